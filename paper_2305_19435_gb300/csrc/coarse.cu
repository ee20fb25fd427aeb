// Cluster mapping (Alg. 1: distances of the query's d_c prefix to every
// centroid, the n_p smallest by (distance, list id)) for short prefixes and
// small n_p, the common AdANNS operating point (d_c <= 64, n_p <= 32).
//
// A CTA takes 32 queries (4 per warp) and streams the centroid table through
// shared memory in chunks, transposed to dimension-major so that lane i reads
// centroids i, i + 32, ... without bank conflicts; each centroid value is used
// by the warp's 4 queries.  Distances are accumulated in the same order and
// form as the general scan kernel (t = q_j - x_j, acc += t * t over j
// ascending), so the two give bit-identical keys.
//
// Each query's running top-32 lives in registers, one key per lane, sorted
// across the warp.  A slot of 32 new candidates is filtered against the
// current n_p-th key; a few survivors are inserted one by one (a shift by one
// lane), many are sorted in registers and merged with a bitonic half-cleaner.
// No shared-memory buffer and no block barrier inside a chunk.
#include "devutil.cuh"
#include "internal.cuh"

namespace adn {
namespace {

constexpr int CM_THREADS = 256;
constexpr int CM_WARPS = CM_THREADS / 32;
constexpr int CM_QPW = 4;                        // queries per warp
constexpr int CM_QPC = CM_WARPS * CM_QPW;        // queries per CTA
constexpr int CM_MAXD = 64;
constexpr int CM_MAXK = 32;

// centroids per chunk: 256 up to d_c = 32, 128 above (keeps the staged chunks small)
inline int coarse_chunk(int d_c) { return d_c <= 32 ? 256 : 128; }

// shared memory: two transposed centroid chunks [d_c][cc + 1] and the CTA's
// query rows [CM_QPC][d_c]
size_t coarse_smem_bytes(int d_c) {
  const int cc = coarse_chunk(d_c);
  return (size_t)2 * d_c * (cc + 1) * 4 + (size_t)CM_QPC * d_c * 4;
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// ascending bitonic sort of one key per lane across the warp (shuffles only)
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v, stride);
      const bool up = (lane & size) == 0;        // direction of this lane's sequence
      const bool lower = (lane & stride) == 0;   // this lane holds the smaller position
      v = (lower == up) ? umin64(o, v) : umax64(o, v);
    }
  }
  return v;
}

// lst: the 32 smallest keys so far, ascending across the lanes.  Adds the
// warp's candidate keys c (one per lane) that beat the k-th entry.
__device__ __forceinline__ void topk_insert(uint64_t &lst, uint64_t c, int k) {
  const int lane = threadIdx.x & 31;
  const uint64_t tau = __shfl_sync(0xffffffffu, lst, k - 1);
  const bool take = c < tau;
  unsigned m = __ballot_sync(0xffffffffu, take);
  if (m == 0) return;
  if (__popc(m) > 4) {
    // sort the survivors, reverse them, keep the lane-wise minimum (the 32
    // smallest of both, as a bitonic sequence) and clean it to ascending order
    uint64_t s = warp_sort32(take ? c : KEY_MAX);
    s = __shfl_sync(0xffffffffu, s, 31 - lane);
    uint64_t v = umin64(lst, s);
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v, stride);
      v = (lane & stride) ? umax64(o, v) : umin64(o, v);
    }
    lst = v;
  } else {
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const uint64_t x = __shfl_sync(0xffffffffu, c, src);
      const int p = __popc(__ballot_sync(0xffffffffu, lst < x));  // its rank in the list
      const uint64_t prev = __shfl_up_sync(0xffffffffu, lst, 1);
      if (lane > p) lst = prev;
      else if (lane == p) lst = x;
    }
  }
}

template <int SLOTS>
__global__ void __launch_bounds__(CM_THREADS) coarse_topk_kernel(
    const float *__restrict__ cent, int ldc, int nlist, int d_c, const float *__restrict__ qc,
    int ldq, int64_t B, int k, uint64_t *__restrict__ out) {
  constexpr int CC = 32 * SLOTS, CCP = CC + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *s_cent = (float *)smem_raw;                    // [2][d_c][CCP]
  float *s_q = s_cent + 2 * d_c * CCP;                  // [CM_QPC][d_c]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q0 = (int64_t)blockIdx.x * CM_QPC;
  for (int e = threadIdx.x; e < CM_QPC * d_c; e += CM_THREADS) {
    const int qi = e / d_c, t = e - qi * d_c;
    s_q[e] = q0 + qi < B ? qc[(q0 + qi) * ldq + t] : 0.f;
  }
  // element e = c * d_c + t of a chunk; this thread's first (c, t) and the
  // step between its elements, so the staging loop needs no division
  const int c_first = (int)threadIdx.x / d_c, t_first = (int)threadIdx.x - c_first * d_c;
  const int c_step = CM_THREADS / d_c, t_step = CM_THREADS - c_step * d_c;
  auto stage = [&](int chunk, int buf) {
    const int c0 = chunk * CC;
    float *dst = s_cent + (size_t)buf * d_c * CCP;
    int c = c_first, t = t_first;
    for (int e = threadIdx.x; e < CC * d_c; e += CM_THREADS) {
      if (c0 + c < nlist) cp_async4(dst + t * CCP + c, cent + (int64_t)(c0 + c) * ldc + t);
      else dst[t * CCP + c] = 0.f;
      c += c_step;
      t += t_step;
      if (t >= d_c) {
        t -= d_c;
        ++c;
      }
    }
    cp_async_commit();
  };
  const int nchunk = (nlist + CC - 1) / CC;
  stage(0, 0);
  cp_async_wait<0>();
  uint64_t lst[CM_QPW];
#pragma unroll
  for (int j = 0; j < CM_QPW; ++j) lst[j] = KEY_MAX;
  __syncthreads();
  const int qb = warp * CM_QPW;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int cur = ch & 1;
    if (ch + 1 < nchunk) stage(ch + 1, cur ^ 1);  // lands while this chunk is scored
    const float *cc = s_cent + (size_t)cur * d_c * CCP;
    float acc[CM_QPW][SLOTS];
#pragma unroll
    for (int j = 0; j < CM_QPW; ++j)
#pragma unroll
      for (int i = 0; i < SLOTS; ++i) acc[j][i] = 0.f;
    for (int t = 0; t < d_c; ++t) {
      float qv[CM_QPW], xv[SLOTS];
#pragma unroll
      for (int j = 0; j < CM_QPW; ++j) qv[j] = s_q[(qb + j) * d_c + t];
#pragma unroll
      for (int i = 0; i < SLOTS; ++i) xv[i] = cc[t * CCP + lane + 32 * i];
#pragma unroll
      for (int j = 0; j < CM_QPW; ++j)
#pragma unroll
        for (int i = 0; i < SLOTS; ++i) {
          const float d = fmaf(-1.f, xv[i], qv[j]);
          acc[j][i] = fmaf(d, d, acc[j][i]);
        }
    }
    const int c0 = ch * CC;
#pragma unroll
    for (int j = 0; j < CM_QPW; ++j)
#pragma unroll
      for (int i = 0; i < SLOTS; ++i) {
        const int c = c0 + lane + 32 * i;
        topk_insert(lst[j], c < nlist ? pack_key(acc[j][i], (uint32_t)c) : KEY_MAX, k);
      }
    cp_async_wait<0>();
    __syncthreads();  // the next chunk has landed; this one is no longer read
  }
#pragma unroll
  for (int j = 0; j < CM_QPW; ++j) {
    const int64_t q = q0 + qb + j;
    if (q < B && lane < k) out[q * k + lane] = lst[j];
  }
}

}  // namespace

// Returns 1 (nothing launched) when the shape is outside the fast path.
int launch_coarse(const float *cent, int ldc, int nlist, int d_c, const float *qc, int ldq,
                  int64_t B, int k, uint64_t *out, cudaStream_t st) {
  if (d_c > CM_MAXD || k > CM_MAXK || d_c < 1 || k < 1 || nlist < k) return 1;
  if (B == 0) return ADANNS_OK;
  const size_t smem = coarse_smem_bytes(d_c);
  const unsigned grid = (unsigned)((B + CM_QPC - 1) / CM_QPC);
  if (coarse_chunk(d_c) == 256) {
    ADN_CUDA(ensure_smem((const void *)coarse_topk_kernel<8>, smem));
    coarse_topk_kernel<8><<<grid, CM_THREADS, smem, st>>>(cent, ldc, nlist, d_c, qc, ldq, B, k, out);
  } else {
    ADN_CUDA(ensure_smem((const void *)coarse_topk_kernel<4>, smem));
    coarse_topk_kernel<4><<<grid, CM_THREADS, smem, st>>>(cent, ldc, nlist, d_c, qc, ldq, B, k, out);
  }
  ADN_LAUNCH("coarse_topk_kernel");
  return ADANNS_OK;
}

}  // namespace adn
