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
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

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

// ---------------------------------------------------------------- tensor-core cluster mapping
// The BF16 products only shortlist: with r_c = c - s_c c~ and r_q = P(q) - s_q q~
// the residuals of the stored low-precision values,
//   P(q).c - (s_q q~).(s_c c~) = P(q).r_c + r_q.c - r_q.r_c,
// so, by Cauchy-Schwarz with |P(q)| <= 1, the approximate distance is within
//   E_q = 2 (R + rho_q |c|max + R rho_q) (1 + 1e-3) + e_rest
// of the exact one (R = max |r_c[0:d_c]|, rho_q = |r_q|; e_rest bounds the FP32
// tensor-core accumulation 2 d_pad 2^-22, the FP32 norm terms 8 (d_c + 2) 2^-24,
// plus 1e-4).  Keys are round(16384 d~) (+-2^-15): every centroid whose key is
// within 2 * 16384 * (2^-15 + E_q) of the k-th smallest key is scored exactly,
// and nothing beyond can be among the k nearest.
namespace adn {
namespace {

constexpr int CT_BM = 128;  // queries per tensor-core tile

// one warp per centroid: BF16 blocks, scale, squared prefix norms, residuals
__global__ void centroid_lowp_kernel(const float *__restrict__ cent, int d_c, int nlist, int nblk,
                                     int ng, __nv_bfloat16 *__restrict__ out,
                                     float *__restrict__ sc, float *__restrict__ n2,
                                     float *__restrict__ rmax, float *__restrict__ maxnorm) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nlist) return;
  const float *src = cent + (int64_t)c * d_c;
  float mx = 0.f;
  for (int j = lane; j < d_c; j += 32) mx = fmaxf(mx, fabsf(src[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float s = mx > 0.f ? mx : 1.f;
  if (lane == 0) sc[c] = s;
  float rseg[NGRAN], xseg[NGRAN];
#pragma unroll
  for (int g = 0; g < NGRAN; ++g) rseg[g] = xseg[g] = 0.f;
  int g = 0;
  for (int j = lane; j < nblk * 64; j += 32) {
    const float v = j < d_c ? src[j] / s : 0.f;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    out[((int64_t)(j >> 6) * nlist + c) * 64 + (j & 63)] = b;
    if (j < d_c) {
      while (g < NGRAN - 1 && j >= kGranDev(g)) ++g;
      const float r = fmaf(-s, __bfloat162float(b), src[j]);
#pragma unroll
      for (int t = 0; t < NGRAN; ++t)
        if (t == g) {
          rseg[t] = fmaf(r, r, rseg[t]);
          xseg[t] = fmaf(src[j], src[j], xseg[t]);
        }
    }
  }
  float rpre = 0.f, xpre = 0.f;
#pragma unroll
  for (int t = 0; t < NGRAN; ++t) {
    float rv = rseg[t], xv = xseg[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rv += __shfl_xor_sync(0xffffffffu, rv, o);
      xv += __shfl_xor_sync(0xffffffffu, xv, o);
    }
    rpre += rv;
    xpre += xv;
    if (lane == 0 && t < ng) {
      n2[(int64_t)t * nlist + c] = xpre;
      atomicMax((int *)(rmax + t), __float_as_int(sqrtf(rpre)));  // non-negative floats order as ints
    }
  }
  if (lane == 0) atomicMax((int *)maxnorm, __float_as_int(sqrtf(xpre)));
}

// query rows P_dc(q) (FP32, zero beyond d_c) -> BF16 tensor-core tiles
// [tile][kb][128 rows][64], the squared norm, the scale and the residual norm
__global__ void coarse_prep_kernel(const float *__restrict__ qc, int ldq, int64_t B, int d_c,
                                   int nkb, int64_t rows, __nv_bfloat16 *__restrict__ tiles,
                                   float *__restrict__ qn2, float *__restrict__ qsc,
                                   float *__restrict__ qrho) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= rows) return;
  const int64_t t = q / CT_BM, r = q - t * CT_BM;
  const bool valid = q < B;
  const float *src = qc + q * ldq;
  float s2 = 0.f, mx = 0.f;
  if (valid)
    for (int j = lane; j < d_c; j += 32) {
      const float v = src[j];
      s2 = fmaf(v, v, s2);
      mx = fmaxf(mx, fabsf(v));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const float s = mx > 0.f ? mx : 1.f;
  float r2 = 0.f;
  for (int j = lane; j < nkb * 64; j += 32) {
    const float v = (valid && j < d_c) ? src[j] / s : 0.f;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    tiles[((t * nkb + (j >> 6)) * CT_BM + r) * 64 + (j & 63)] = b;
    if (valid && j < d_c) {
      const float e = fmaf(-s, __bfloat162float(b), src[j]);
      r2 = fmaf(e, e, r2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if (valid && lane == 0) {
    qn2[q] = s2;
    qsc[q] = s;
    qrho[q] = sqrtf(r2);
  }
}

// the tensor-core scan's work description: every tile is (centroid list,
// 128 consecutive queries); pair p = query p, its key segment at p * npad
__global__ void coarse_tiles_kernel(int64_t B, int ntiles, int64_t npad, int32_t *__restrict__ tl,
                                    int32_t *__restrict__ tb, int32_t *__restrict__ tc,
                                    int32_t *__restrict__ pair_out, int64_t *__restrict__ pbase,
                                    int *__restrict__ ntiles_dev, int *__restrict__ counter) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ntiles) {
    tl[i] = 0;
    tb[i] = (int32_t)(i * CT_BM);
    tc[i] = (int32_t)min((int64_t)CT_BM, B - i * CT_BM);
  }
  if (i < B) {
    pair_out[i] = (int32_t)i;
    pbase[i] = i * npad;
  }
  if (i == 0) {
    *ntiles_dev = ntiles;
    *counter = 0;
  }
}

// One warp per query (k <= 32): the top byte of the k-th smallest key (one
// radix pass over the key row) gives an upper bound of that key, the end of
// its 256-key bucket, and the threshold above it; the centroids under the
// threshold (at most CP_CAND, collected in list order) are scored exactly, one
// per lane, with the same arithmetic as the FP32 kernels, and the k nearest by
// (distance, list id) are written.  More candidates than CP_CAND (a loose
// bound) take a second pass that scores them while streaming the row.
constexpr int CP_WARPS = 8;
constexpr int CP_CAND = 96;

__global__ void __launch_bounds__(CP_WARPS * 32) coarse_pick_kernel(
    const uint16_t *__restrict__ keys, int64_t npad, int nlist, const float *__restrict__ qc,
    int ldq, int d_c, const float *__restrict__ cent, int ldc, const float *__restrict__ qrho,
    float rmax, float cmax, float e_rest, int64_t B, int k, uint64_t *__restrict__ out) {
  __shared__ float s_q[CP_WARPS][CM_MAXD];
  __shared__ int s_hist[CP_WARPS][256];
  __shared__ int s_sh[CP_WARPS][2];
  __shared__ int s_cand[CP_WARPS][CP_CAND];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * CP_WARPS + warp;
  if (q >= B) return;
  for (int j = lane; j < d_c; j += 32) s_q[warp][j] = qc[q * ldq + j];
  const uint16_t *kq = keys + q * npad;
  int below, neq;
  const uint32_t kth = (warp_radix_kth<1>(
                            nlist, k, [&](int i) -> uint32_t { return __ldg(kq + i) >> 8; },
                            s_hist[warp], s_sh[warp], below, neq)
                        << 8) | 0xFFu;
  const double rq = (double)qrho[q];
  const double E = 2.0 * (rmax + rq * cmax + rmax * rq) * (1.0 + 1e-3) + e_rest;
  const uint32_t thr = kth + (uint32_t)ceil(2.0 * 16384.0 * (ldexp(1.0, -15) + E)) + 1u;
  auto score = [&](int c) -> uint64_t {
    const float *x = cent + (int64_t)c * ldc;
    float acc = 0.f;
#pragma unroll 8
    for (int t = 0; t < d_c; ++t) {
      const float d = fmaf(-1.f, __ldg(x + t), s_q[warp][t]);
      acc = fmaf(d, d, acc);
    }
    return pack_key(acc, (uint32_t)c);
  };
  // candidates under the threshold, in list order
  int nc = 0;
  for (int c0 = 0; c0 < nlist; c0 += 32) {
    const int c = c0 + lane;
    const bool in = c < nlist && __ldg(kq + c) <= thr;
    const unsigned m = __ballot_sync(0xffffffffu, in);
    const int p = nc + __popc(m & lanemask_lt());
    if (in && p < CP_CAND) s_cand[warp][p] = c;
    nc += __popc(m);
  }
  __syncwarp();
  uint64_t best = KEY_MAX;
  if (nc <= CP_CAND) {
    for (int j0 = 0; j0 < nc; j0 += 32) {
      const int j = j0 + lane;
      topk_insert(best, j < nc ? score(s_cand[warp][j]) : KEY_MAX, k);
    }
  } else {
    for (int c0 = 0; c0 < nlist; c0 += 32) {
      const int c = c0 + lane;
      topk_insert(best, c < nlist && __ldg(kq + c) <= thr ? score(c) : KEY_MAX, k);
    }
  }
  if (lane < k) out[q * k + lane] = best;
}

// One CTA per query, for 32 < k <= 1,024 over at most CPB_MAXLIST centroids:
// the k-th smallest 16-bit key (two-digit radix select on the query's key
// row staged in shared memory) gives the same threshold as above; every
// centroid under it gets its exact FP32 distance, the rest +inf bits; a
// four-digit radix select on those bits with ties to the lowest list id picks
// the k nearest, which one warp sorts by (distance, list id).
constexpr int CPB_THREADS = 256;
constexpr int CPB_MAXK = 1024;
constexpr int CPB_MAXLIST = 16384;

__global__ void __launch_bounds__(CPB_THREADS) coarse_pick_block_kernel(
    const uint16_t *__restrict__ keys, int64_t npad, int nlist, const float *__restrict__ qc,
    int ldq, int d_c, const float *__restrict__ cent, int ldc, const float *__restrict__ qrho,
    float rmax, float cmax, float e_rest, int k, uint64_t *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *cd = (uint32_t *)smem;          // [nlist] exact distance bits
  uint16_t *k16 = (uint16_t *)(cd + nlist);  // [nlist] tensor-core keys
  __shared__ float s_q[CM_MAXD];
  __shared__ int hist[256], sh[2], wsum[CPB_THREADS / 32];
  __shared__ int s_lt;
  __shared__ uint64_t s_out[CPB_MAXK];
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int j = tid; j < d_c; j += CPB_THREADS) s_q[j] = qc[q * ldq + j];
  const uint16_t *kq = keys + q * npad;
  for (int c = tid; c < nlist; c += CPB_THREADS) k16[c] = kq[c];
  if (tid == 0) s_lt = 0;
  __syncthreads();
  int below, neq;
  const uint32_t kth = block_radix_kth<CPB_THREADS, 2>(
      nlist, k, [&](int i) -> uint32_t { return k16[i]; }, hist, sh, &below, &neq);
  const double rq = (double)qrho[q];
  const double E = 2.0 * (rmax + rq * cmax + rmax * rq) * (1.0 + 1e-3) + e_rest;
  const uint32_t thr = kth + (uint32_t)ceil(2.0 * 16384.0 * (ldexp(1.0, -15) + E)) + 1u;
  for (int c = tid; c < nlist; c += CPB_THREADS) {
    uint32_t v = 0xFFFFFFFFu;
    if (k16[c] <= thr) {
      const float *x = cent + (int64_t)c * ldc;
      float acc = 0.f;
      for (int t = 0; t < d_c; ++t) {
        const float d = fmaf(-1.f, x[t], s_q[t]);
        acc = fmaf(d, d, acc);
      }
      v = __float_as_uint(acc);
    }
    cd[c] = v;
  }
  __syncthreads();
  const uint32_t T = block_radix_kth<CPB_THREADS, 4>(
      nlist, k, [&](int i) -> uint32_t { return cd[i]; }, hist, sh, &below, &neq);
  for (int c = tid; c < nlist; c += CPB_THREADS)
    if (cd[c] < T) s_out[atomicAdd(&s_lt, 1)] = ((uint64_t)cd[c] << 32) | (uint32_t)c;
  // the k - below lowest list ids among the centroids at distance T
  const int need = k - below;
  int base = 0;
  for (int c0 = 0; c0 < nlist && base < need; c0 += CPB_THREADS) {
    const int c = c0 + tid;
    const bool eq = c < nlist && cd[c] == T;
    const unsigned b = __ballot_sync(0xffffffffu, eq);
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    int before = base, tot = 0;
    for (int w = 0; w < CPB_THREADS / 32; ++w) {
      if (w < warp) before += wsum[w];
      tot += wsum[w];
    }
    before += __popc(b & lanemask_lt());
    if (eq && before < need) s_out[below + before] = ((uint64_t)T << 32) | (uint32_t)c;
    __syncthreads();
    base += tot;
  }
  __syncthreads();
  if (warp == 0) {
    warp_sort(s_out, k);
    for (int r = lane; r < k; r += 32) out[q * k + r] = s_out[r];
  }
}

}  // namespace

int build_centroid_lowp(adanns_index *x, cudaStream_t st) {
  if (x->metric != ADANNS_METRIC_L2_PREFIXNORM || x->nlist < 256) return ADANNS_OK;
  const int nblk = (x->d_c + 63) / 64;
  int ng = 0;
  for (int g = 0; g < NGRAN; ++g)
    if (kGran[g] <= x->d_c) ng = g + 1;
  void *lowp = nullptr;
  float *sc = nullptr, *n2 = nullptr, *tmp = nullptr;
  if (cudaMalloc(&lowp, (size_t)nblk * x->nlist * 64 * 2) != cudaSuccess ||
      cudaMalloc(&sc, sizeof(float) * x->nlist) != cudaSuccess ||
      cudaMalloc(&n2, sizeof(float) * x->nlist * std::max(ng, 1)) != cudaSuccess ||
      cudaMalloc(&tmp, sizeof(float) * (NGRAN + 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(lowp);
    cudaFree(sc);
    cudaFree(n2);
    cudaFree(tmp);
    return fail(ADANNS_ERR_OOM, "centroid low-precision copy allocation failed");
  }
  ADN_CUDA(cudaMemsetAsync(tmp, 0, sizeof(float) * (NGRAN + 1), st));
  centroid_lowp_kernel<<<(unsigned)((x->nlist + 7) / 8), 256, 0, st>>>(
      x->centroids, x->d_c, x->nlist, nblk, ng, (__nv_bfloat16 *)lowp, sc, n2, tmp, tmp + NGRAN);
  ADN_LAUNCH("centroid_lowp_kernel");
  float h[NGRAN + 1];
  cudaError_t e = cudaMemcpyAsync(h, tmp, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) {
    cudaFree(lowp);
    cudaFree(sc);
    cudaFree(n2);
    return cuda_fail(e, "centroid low-precision copy");
  }
  x->cent_low = lowp;
  x->cent_low_blocks = nblk;
  x->cent_sc = sc;
  x->cent_n2 = n2;
  for (int g = 0; g < NGRAN; ++g) x->cent_rmax[g] = h[g];
  x->cent_maxnorm = h[NGRAN];
  return ADANNS_OK;
}

int launch_mma_scan(const void *qtiles, int64_t qrows, const void *xlow, int64_t xrows,
                    const MmaScanArgs &a, cudaStream_t st);

int launch_coarse_tc(const adanns_index *idx, const float *qc, int ldq, int64_t B, int d_c, int k,
                     uint64_t *out, cudaStream_t st) {
  // small tables stay on the FP32 kernels (they are cheap there, and the
  // tensor-core tile reads 256 centroid rows at a time)
  if (!option(ADANNS_OPT_COARSE_TC) || !idx->cent_low || d_c > CM_MAXD || k > idx->nlist ||
      idx->nlist < 256 || k > CPB_MAXK || (k > CM_MAXK && idx->nlist > CPB_MAXLIST))
    return 1;
  if (B == 0) return ADANNS_OK;
  const int gi = gran_index(d_c);
  if (gi < 0) return 1;
  const int nlist = idx->nlist, nkb = (d_c + 63) / 64;
  const int ntiles = (int)((B + CT_BM - 1) / CT_BM);
  const int64_t rows = (int64_t)ntiles * CT_BM;
  const int64_t npad = (nlist + 7) & ~7;
  Scratch s(st);
  __nv_bfloat16 *tiles;
  float *qn2, *qsc, *qrho;
  uint16_t *keys;
  int32_t *tl, *tb, *tc, *pair_out;
  int64_t *pbase;
  int *ntiles_dev, *counter;
  int rc;
  if ((rc = s.get(&tiles, (size_t)rows * nkb * 64)) || (rc = s.get(&qn2, B)) ||
      (rc = s.get(&qsc, B)) || (rc = s.get(&qrho, B)) || (rc = s.get(&keys, (size_t)B * npad)) ||
      (rc = s.get(&tl, ntiles)) || (rc = s.get(&tb, ntiles)) || (rc = s.get(&tc, ntiles)) ||
      (rc = s.get(&pair_out, B)) || (rc = s.get(&pbase, B)) || (rc = s.get(&ntiles_dev, 1)) ||
      (rc = s.get(&counter, 1)))
    return rc;
  const int64_t nfill = std::max<int64_t>(B, ntiles);
  coarse_tiles_kernel<<<(unsigned)((nfill + 255) / 256), 256, 0, st>>>(
      B, ntiles, npad, tl, tb, tc, pair_out, pbase, ntiles_dev, counter);
  ADN_LAUNCH("coarse_tiles_kernel");
  coarse_prep_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(qc, ldq, B, d_c, nkb, rows, tiles,
                                                                 qn2, qsc, qrho);
  ADN_LAUNCH("coarse_prep_kernel");
  MmaScanArgs m{};
  m.tile_list = tl;
  m.tile_beg = tb;
  m.tile_cnt = tc;
  m.ntiles_dev = ntiles_dev;
  m.list_off = idx->cent_off;
  m.pair_out = pair_out;
  m.pbase = pbase;
  m.cx = idx->cent_sc;
  m.x2 = idx->cent_n2 + (int64_t)gi * nlist;
  m.qn2 = qn2;
  m.qsc = qsc;
  m.nprobe = 1;
  m.nkb = nkb;
  m.d_blocks = idx->cent_low_blocks;
  m.cand = keys;
  m.err = idx->dev_err;
  m.tile_counter = counter;
  m.fp8 = 0;
  if ((rc = launch_mma_scan(tiles, rows * nkb, idx->cent_low,
                            (int64_t)nlist * idx->cent_low_blocks, m, st)))
    return rc;
  const float e_rest = (float)(2.0 * nkb * 64 * std::ldexp(1.0, -22) +
                               8.0 * (d_c + 2) * std::ldexp(1.0, -24) + 1e-4);
  if (k <= CM_MAXK) {
    coarse_pick_kernel<<<(unsigned)((B + CP_WARPS - 1) / CP_WARPS), CP_WARPS * 32, 0, st>>>(
        keys, npad, nlist, qc, ldq, d_c, idx->centroids, idx->d_c, qrho,
        idx->cent_rmax[gi] * 1.001f, idx->cent_maxnorm * 1.001f, e_rest, B, k, out);
    ADN_LAUNCH("coarse_pick_kernel");
  } else {
    const size_t sm = (size_t)nlist * 6;
    ADN_CUDA(ensure_smem((const void *)coarse_pick_block_kernel, sm));
    coarse_pick_block_kernel<<<(unsigned)B, CPB_THREADS, sm, st>>>(
        keys, npad, nlist, qc, ldq, d_c, idx->centroids, idx->d_c, qrho,
        idx->cent_rmax[gi] * 1.001f, idx->cent_maxnorm * 1.001f, e_rest, k, out);
    ADN_LAUNCH("coarse_pick_block_kernel");
  }
  return ADANNS_OK;
}

int run_coarse(const adanns_index *idx, const float *qc, int ldq, int64_t B, int d_c, int k,
               uint64_t *out, int *counter, cudaStream_t st) {
  int rc = launch_coarse_tc(idx, qc, ldq, B, d_c, k, out, st);
  if (rc == 1) rc = launch_coarse(idx->centroids, idx->d_c, idx->nlist, d_c, qc, ldq, B, k, out, st);
  if (rc == 1) {
    // the general scan over the prefix-major centroid table (one list)
    ScanArgs c{};
    c.xpm = idx->cent_pm;
    c.d_pad = idx->dc_pad;  // stored centroid width; d_c <= built d_c (IVF-D)
    c.dims = d_c;
    c.list_off = idx->cent_off;
    c.qn = qc;
    c.ldq = ldq;
    c.nq = (int)B;
    c.counter = counter;
    c.k = k;
    c.out_keys = out;
    rc = launch_scan_f32(c, st);
  }
  return rc;
}

}  // namespace adn
