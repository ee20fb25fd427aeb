// Inverted lists partitioned over several GPUs: each GPU holds the lists it
// owns (with the replicated centroids, so every GPU probes the same lists)
// and answers the whole batch over them; the per-GPU top-k are exchanged and
// merged per query.  The two device steps of that exchange live here:
//   adanns_map_ids      local row ids of a shard -> global database ids
//   adanns_merge_shards G sorted per-shard top-k rows -> one top-k per query
// The exchange itself (who sends which rows where) is the caller's, over any
// transport; the merge order is (distance, id) ascending, the same order as a
// single-GPU search, so the merged result equals the unpartitioned search.
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {
namespace {

constexpr int SH_PER_LANE = ADANNS_MAX_SHARDS / 32;
constexpr int SH_WPB = 8;

__global__ void map_ids_kernel(const int64_t *__restrict__ map, int64_t n_map,
                               int64_t *__restrict__ ids, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = ids[i];
    if (v < 0) continue;
    ids[i] = v < n_map ? map[v] : -1;
  }
}

__device__ __forceinline__ uint64_t shard_key(const int64_t *ids, const float *dist, int64_t o) {
  const int64_t id = ids[o];
  if (id < 0 || id >= 0xffffffffll) return KEY_MAX;
  return pack_key(dist[o], (uint32_t)id);
}

// One warp per query.  Lane l holds the heads of shards l, l + 32, ...; each
// of the k steps takes the smallest head over the warp (lowest lane on a
// tie, which only equal (distance, id) pairs from two shards can produce) and
// advances that shard.
__global__ void __launch_bounds__(SH_WPB * 32) merge_shards_kernel(
    const int64_t *__restrict__ ids, const float *__restrict__ dist, int G, int64_t B, int k,
    int64_t *__restrict__ out_ids, float *__restrict__ out_dist) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * SH_WPB + warp;
  if (q >= B) return;
  int pos[SH_PER_LANE];
  uint64_t head[SH_PER_LANE];
#pragma unroll
  for (int j = 0; j < SH_PER_LANE; ++j) {
    const int s = lane + 32 * j;
    pos[j] = 0;
    head[j] = s < G ? shard_key(ids, dist, ((int64_t)s * B + q) * k) : KEY_MAX;
  }
  for (int r = 0; r < k; ++r) {
    uint64_t best = KEY_MAX;
    int bj = 0;
#pragma unroll
    for (int j = 0; j < SH_PER_LANE; ++j)
      if (head[j] < best) {
        best = head[j];
        bj = j;
      }
    const uint64_t wbest = warp_min_u64(best);
    if (wbest == KEY_MAX) {
      for (int t = r + lane; t < k; t += 32) {
        out_ids[q * k + t] = -1;
        out_dist[q * k + t] = __int_as_float(0x7f800000);
      }
      return;
    }
    const unsigned m = __ballot_sync(0xffffffffu, best == wbest);
    if (lane == __ffs(m) - 1) {
#pragma unroll
      for (int j = 0; j < SH_PER_LANE; ++j)
        if (j == bj) {
          const int s = lane + 32 * j;
          ++pos[j];
          head[j] = pos[j] < k ? shard_key(ids, dist, ((int64_t)s * B + q) * k + pos[j]) : KEY_MAX;
        }
      out_ids[q * k + r] = (int64_t)(uint32_t)(wbest & 0xffffffffu);
      out_dist[q * k + r] = __uint_as_float((uint32_t)(wbest >> 32));
    }
  }
}

}  // namespace
}  // namespace adn

using namespace adn;

extern "C" int adanns_map_ids(const int64_t *map, int64_t n_map, int64_t *ids, int64_t count,
                              void *cuda_stream) {
  if (count < 0 || n_map < 0) return fail(ADANNS_ERR_ARG, "negative size");
  if (count == 0) return ADANNS_OK;
  if (!ids || (n_map > 0 && !map)) return fail(ADANNS_ERR_ARG, "NULL argument");
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)num_sms() * 8);
  map_ids_kernel<<<(unsigned)blocks, 256, 0, st>>>(map, n_map, ids, count);
  ADN_LAUNCH("map_ids_kernel");
  return ADANNS_OK;
}

extern "C" int adanns_merge_shards(const int64_t *ids, const float *dist, int G, int64_t B, int k,
                                   int64_t *out_ids, float *out_dist, void *cuda_stream) {
  if (G < 1 || G > ADANNS_MAX_SHARDS)
    return fail(ADANNS_ERR_ARG, "need 1 <= G <= " + std::to_string(ADANNS_MAX_SHARDS));
  if (k < 1 || k > 1024) return fail(ADANNS_ERR_ARG, "need 1 <= k <= 1024");
  if (B < 0 || B > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad batch size");
  if (B == 0) return ADANNS_OK;
  if (!ids || !dist || !out_ids || !out_dist) return fail(ADANNS_ERR_ARG, "NULL argument");
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  merge_shards_kernel<<<(unsigned)((B + SH_WPB - 1) / SH_WPB), SH_WPB * 32, 0, st>>>(
      ids, dist, G, B, k, out_ids, out_dist);
  ADN_LAUNCH("merge_shards_kernel");
  return ADANNS_OK;
}
