// Cluster mapping (Alg. 1: distances of the query's d_c prefix to every
// centroid, the n_p smallest by (distance, list id)) for short prefixes and
// small n_p, the common AdANNS operating point (d_c <= 64).
//
// A CTA takes 32 queries (4 per warp) and streams the centroid table through
// shared memory in chunks of 256, transposed to dimension-major so that lane
// i reads centroids i, i + 32, ... without bank conflicts; each centroid value
// is used by the warp's 4 queries.  Distances are accumulated in the same
// order and form as the general scan kernel (t = q_j - x_j, acc += t * t over
// j ascending), so the two give bit-identical keys.  Each query keeps its
// candidates in a small shared buffer: a candidate enters only if it beats the
// query's current n_p-th key, and the warp sorts and trims the buffer when the
// next round could overflow it.  Only warp-level synchronisation is used
// inside a chunk.
#include "devutil.cuh"
#include "internal.cuh"

namespace adn {
namespace {

constexpr int CM_THREADS = 256;
constexpr int CM_WARPS = CM_THREADS / 32;
constexpr int CM_QPW = 4;                        // queries per warp
constexpr int CM_QPC = CM_WARPS * CM_QPW;        // queries per CTA
constexpr int CM_CC = 256;                       // centroids per chunk
constexpr int CM_CCP = CM_CC + 1;                // padded row of the transposed chunk
constexpr int CM_MAXD = 64;
constexpr int CM_MAXK = 64;
constexpr int CM_ROUND = 64;                     // candidates a query can gain per round
constexpr int CM_CAP = CM_MAXK + CM_ROUND;

// shared memory, sized by d_c: two transposed centroid chunks [d_c][CM_CCP],
// the CTA's query rows [CM_QPC][d_c], the candidate buffers [CM_QPC][CM_CAP]
size_t coarse_smem_bytes(int d_c) {
  return (size_t)2 * d_c * CM_CCP * 4 + (size_t)CM_QPC * d_c * 4 + (size_t)CM_QPC * CM_CAP * 8;
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

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
      const uint64_t mn = o < v ? o : v, mx = o < v ? v : o;
      v = (lower == up) ? mn : mx;
    }
  }
  return v;
}

__global__ void __launch_bounds__(CM_THREADS) coarse_topk_kernel(
    const float *__restrict__ cent, int ldc, int nlist, int d_c, const float *__restrict__ qc,
    int ldq, int64_t B, int k, uint64_t *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t *s_buf = (uint64_t *)smem_raw;                     // [CM_QPC][CM_CAP]
  float *s_cent = (float *)(s_buf + CM_QPC * CM_CAP);         // [2][d_c][CM_CCP]
  float *s_q = s_cent + 2 * d_c * CM_CCP;                     // [CM_QPC][d_c]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q0 = (int64_t)blockIdx.x * CM_QPC;
  // this CTA's query rows
  for (int e = threadIdx.x; e < CM_QPC * d_c; e += CM_THREADS) {
    const int qi = e / d_c, t = e - qi * d_c;
    s_q[e] = q0 + qi < B ? qc[(q0 + qi) * ldq + t] : 0.f;
  }
  // chunk of CM_CC centroids, transposed (4-byte asynchronous copies)
  // element e = c * d_c + t of a chunk; this thread's first (c, t) and the
  // step between its elements, so the loop needs no division
  const int c_first = (int)threadIdx.x / d_c, t_first = (int)threadIdx.x - c_first * d_c;
  const int c_step = CM_THREADS / d_c, t_step = CM_THREADS - c_step * d_c;
  auto stage = [&](int chunk, int buf) {
    const int c0 = chunk * CM_CC;
    float *dst = s_cent + (size_t)buf * d_c * CM_CCP;
    int c = c_first, t = t_first;
    for (int e = threadIdx.x; e < CM_CC * d_c; e += CM_THREADS) {
      if (c0 + c < nlist) cp_async4(dst + t * CM_CCP + c, cent + (int64_t)(c0 + c) * ldc + t);
      else dst[t * CM_CCP + c] = 0.f;
      c += c_step;
      t += t_step;
      if (t >= d_c) {
        t -= d_c;
        ++c;
      }
    }
    cp_async_commit();
  };
  const int nchunk = (nlist + CM_CC - 1) / CM_CC;
  stage(0, 0);
  cp_async_wait<0>();
  int n[CM_QPW];
  uint64_t tau[CM_QPW];
#pragma unroll
  for (int j = 0; j < CM_QPW; ++j) {
    n[j] = 0;
    tau[j] = KEY_MAX;
  }
  __syncthreads();
  for (int ch = 0; ch < nchunk; ++ch) {
    const int cur = ch & 1;
    if (ch + 1 < nchunk) stage(ch + 1, cur ^ 1);  // lands while this chunk is scored
    const float *cc = s_cent + (size_t)cur * d_c * CM_CCP;
    float acc[CM_QPW][8];
#pragma unroll
    for (int j = 0; j < CM_QPW; ++j)
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[j][i] = 0.f;
    const int qb = warp * CM_QPW;
    for (int t = 0; t < d_c; ++t) {
      float qv[CM_QPW], xv[8];
#pragma unroll
      for (int j = 0; j < CM_QPW; ++j) qv[j] = s_q[(qb + j) * d_c + t];
#pragma unroll
      for (int i = 0; i < 8; ++i) xv[i] = cc[t * CM_CCP + lane + 32 * i];
#pragma unroll
      for (int j = 0; j < CM_QPW; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float d = fmaf(-1.f, xv[i], qv[j]);
          acc[j][i] = fmaf(d, d, acc[j][i]);
        }
    }
    const int c0 = ch * CM_CC;
#pragma unroll
    for (int j = 0; j < CM_QPW; ++j) {
      uint64_t *b = s_buf + (size_t)(qb + j) * CM_CAP;
      int r0 = 0;
      if (ch == 0 && k <= 32) {
        // seed: the k smallest of the chunk's first 32 candidates, sorted in
        // registers, become the buffer and their k-th key the threshold
        const int c = lane;
        const uint64_t key = c < nlist ? pack_key(acc[j][0], (uint32_t)c) : KEY_MAX;
        const uint64_t v = warp_sort32(key);
        if (lane < k) b[lane] = v;
        n[j] = min(k, min(nlist, 32));
        tau[j] = __shfl_sync(0xffffffffu, v, k - 1);
        if (n[j] < k) tau[j] = KEY_MAX;
        __syncwarp();
        r0 = 1;
      }
#pragma unroll
      for (int r = 0; r < 8; r += 2) {
        // one round: up to 64 new candidates for this query
#pragma unroll
        for (int i = r; i < r + 2; ++i) {
          if (i < r0) continue;  // slot 0 of the first chunk seeded the buffer
          const int c = c0 + lane + 32 * i;
          const uint64_t key = c < nlist ? pack_key(acc[j][i], (uint32_t)c) : KEY_MAX;
          const bool take = key < tau[j];
          const unsigned m = __ballot_sync(0xffffffffu, take);
          if (take) b[n[j] + __popc(m & lanemask_lt())] = key;
          n[j] += __popc(m);
        }
        const bool last = ch == nchunk - 1 && r == 6;
        if (n[j] > CM_CAP - CM_ROUND || (last && n[j] > 0)) {
          __syncwarp();
          warp_sort(b, n[j]);
          if (n[j] > k) n[j] = k;
          if (n[j] == k) tau[j] = b[k - 1];
          __syncwarp();
        }
      }
    }
    cp_async_wait<0>();
    __syncthreads();  // the next chunk has landed; this one is no longer read
  }
#pragma unroll
  for (int j = 0; j < CM_QPW; ++j) {
    const int64_t q = q0 + warp * CM_QPW + j;
    if (q >= B) continue;
    const uint64_t *b = s_buf + (size_t)(warp * CM_QPW + j) * CM_CAP;
    for (int r = lane; r < k; r += 32) out[q * k + r] = r < n[j] ? b[r] : KEY_MAX;
  }
}

}  // namespace

// Returns 1 (nothing launched) when the shape is outside the fast path.
int launch_coarse(const float *cent, int ldc, int nlist, int d_c, const float *qc, int ldq,
                  int64_t B, int k, uint64_t *out, cudaStream_t st) {
  if (d_c > CM_MAXD || k > CM_MAXK || d_c < 1 || k < 1 || nlist < k) return 1;
  if (B == 0) return ADANNS_OK;
  const size_t smem = coarse_smem_bytes(d_c);
  ADN_CUDA(ensure_smem((const void *)coarse_topk_kernel, smem));
  coarse_topk_kernel<<<(unsigned)((B + CM_QPC - 1) / CM_QPC), CM_THREADS, smem, st>>>(
      cent, ldc, nlist, d_c, qc, ldq, B, k, out);
  ADN_LAUNCH("coarse_topk_kernel");
  return ADANNS_OK;
}

}  // namespace adn
