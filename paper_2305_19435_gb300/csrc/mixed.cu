// Mixed-precision AdANNS-IVF search: BF16 / FP8-E4M3 storage with a per-vector
// FP32 scale, tensor-core approximate scan, per-query top-k' selection and the
// exact FP32 rerank of the k' shortlist at d_s (Sec. 4.3 shortlist-rerank; the
// shortlist size k' is the caller's rerank_k, 4k in the benchmark).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {

int launch_rerank(const int64_t *cand, int kr, int64_t B, const float *qs, int ldq, int d_s,
                  const adanns_index *idx, const float *mscale, int k, int64_t *out_ids,
                  float *out_dist, cudaStream_t st);
// cand: B x kr shortlisted candidates as (list << 32 | member position), -1 padding
int launch_rerank_lists(const int64_t *cand, int kr, int64_t B, const float *qs, int ldq, int d_s,
                        const adanns_index *idx, const float *mscale, int k, int64_t *out_ids,
                        float *out_dist, cudaStream_t st);

// ---------------------------------------------------------------- storage
// Member p (list order) of list l: s_x = max_j |x_j| / R (R = 448 for FP8-E4M3,
// 1 for BF16; 1 for a zero vector); element j of block b is stored at
// ((off_l * nblk + b * n_l + m) * epb + j % epb), value x_j / s_x rounded.
// It also folds, per granularity g, nu_g(p) * |(x - s_x x~)[0:g]| (the exact
// residual of the stored values, computed with one rounding per coordinate)
// into rmax[g] by an atomic maximum.
__global__ void quantize_kernel(const float *__restrict__ x, int d, const int64_t *__restrict__ list_off,
                                const int32_t *__restrict__ list_ids,
                                const int32_t *__restrict__ assign, int64_t N, int fp8, int nblk,
                                unsigned char *__restrict__ out, float *__restrict__ sx,
                                const float *__restrict__ invn, int ng, float *__restrict__ rmax) {
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= N) return;
  const int id = list_ids[p];
  const int l = assign[id];
  const int64_t off = list_off[l];
  const int64_t nl = list_off[l + 1] - off;
  const int64_t m = p - off;
  const float *src = x + (int64_t)id * d;
  float mx = 0.f;
  for (int j = lane; j < d; j += 32) mx = fmaxf(mx, fabsf(src[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float R = fp8 ? 448.f : 1.f;
  const float s = mx > 0.f ? mx / R : 1.f;
  if (lane == 0) sx[p] = s;
  const int epb = fp8 ? 128 : 64;
  float seg[NGRAN];  // this lane's squared residuals per granularity segment
#pragma unroll
  for (int g = 0; g < NGRAN; ++g) seg[g] = 0.f;
  int g = 0;
  for (int j = lane; j < nblk * epb; j += 32) {
    const float v = j < d ? src[j] / s : 0.f;
    const int b = j / epb, e = j - b * epb;
    const int64_t o = ((off * nblk + b * nl + m) * epb + e);
    float back;
    if (fp8) {
      const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
      out[o] = (unsigned char)c;
      back = __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3)));
    } else {
      const __nv_bfloat16 c = __float2bfloat16_rn(v);
      ((__nv_bfloat16 *)out)[o] = c;
      back = __bfloat162float(c);
    }
    if (j < d) {
      while (g < NGRAN - 1 && j >= kGranDev(g)) ++g;
      const float r = fmaf(-s, back, src[j]);
#pragma unroll
      for (int t = 0; t < NGRAN; ++t)
        if (t == g) seg[t] = fmaf(r, r, seg[t]);
    }
  }
  float pre = 0.f;
#pragma unroll
  for (int t = 0; t < NGRAN; ++t) {
    float v = seg[t];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
    pre += v;
    if (lane == 0 && t < ng) {
      const float rel = sqrtf(pre) * invn[(int64_t)t * N + p];
      atomicMax((int *)(rmax + t), __float_as_int(rel));  // non-negative floats order as ints
    }
  }
}

// cx[g][p] = s_x[p] * invn[g][p]
__global__ void lowp_scale_kernel(const float *__restrict__ sx, const float *__restrict__ invn,
                                  int64_t N, int ng, float *__restrict__ cx) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * ng) return;
  cx[e] = sx[e % N] * invn[e];
}

int build_lowp(adanns_index *x, const float *db, int which, cudaStream_t st) {
  const int fp8 = which == 1;
  const int epb = fp8 ? 128 : 64;
  const int nblk = (x->d + epb - 1) / epb;
  const size_t elems = (size_t)x->N * nblk * epb;
  const size_t bytes = elems * (fp8 ? 1 : 2);
  void *store = nullptr;
  float *sx = nullptr, *cx = nullptr, *rmax = nullptr;
  if (cudaMalloc(&store, bytes + 256) != cudaSuccess || cudaMalloc(&sx, sizeof(float) * x->N) != cudaSuccess ||
      cudaMalloc(&cx, sizeof(float) * (size_t)x->N * std::max(x->ng, 1)) != cudaSuccess ||
      cudaMalloc(&rmax, sizeof(float) * NGRAN) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(store);
    cudaFree(sx);
    cudaFree(cx);
    cudaFree(rmax);
    return fail(ADANNS_ERR_OOM, "low-precision storage allocation failed");
  }
  ADN_CUDA(cudaMemsetAsync(rmax, 0, sizeof(float) * NGRAN, st));
  quantize_kernel<<<(unsigned)((x->N + 7) / 8), 256, 0, st>>>(
      db, x->d, x->list_off, x->list_ids, x->assign, x->N, fp8, nblk, (unsigned char *)store, sx,
      x->invn, x->ng, rmax);
  ADN_LAUNCH("quantize_kernel");
  {
    float h[NGRAN];
    cudaError_t e = cudaMemcpyAsync(h, rmax, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(rmax);
    if (e != cudaSuccess) return cuda_fail(e, "quantisation residual");
    for (int g = 0; g < NGRAN; ++g) x->lowp_rmax[which][g] = h[g];
  }
  const int64_t ne = x->N * (int64_t)x->ng;
  if (ne > 0) {
    lowp_scale_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(sx, x->invn, x->N, x->ng, cx);
    ADN_LAUNCH("lowp_scale_kernel");
  }
  x->lowp[which] = store;
  x->lowp_blocks[which] = nblk;
  x->lowp_sx[which] = sx;
  x->lowp_cx[which] = cx;
  return ADANNS_OK;
}

// ---------------------------------------------------------------- queries
// Per query (one warp): |P_ds(q)|^2, s_q = max|q| / R, and the low-precision
// row q / s_q (nkb blocks of epb elements, zero beyond d_s).
__global__ void prep_lowp_kernel(const float *__restrict__ qs, int ldq, int64_t B, int d_s,
                                 int fp8, int nkb, unsigned char *__restrict__ out,
                                 float *__restrict__ qn2, float *__restrict__ qsc,
                                 float *__restrict__ qrho) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= B) return;
  const float *src = qs + q * ldq;
  float s2 = 0.f, mx = 0.f;
  for (int j = lane; j < d_s; j += 32) {
    const float v = src[j];
    s2 = fmaf(v, v, s2);
    mx = fmaxf(mx, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const float R = fp8 ? 448.f : 1.f;
  const float s = mx > 0.f ? mx / R : 1.f;
  if (lane == 0) {
    qn2[q] = s2;
    qsc[q] = s;
  }
  const int epb = fp8 ? 128 : 64;
  const int len = nkb * epb;
  float r2 = 0.f;  // |P(q) - s_q q~|^2: the query's own quantisation residual
  for (int j = lane; j < len; j += 32) {
    const float v = j < d_s ? src[j] / s : 0.f;
    float back;
    if (fp8) {
      const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
      out[q * len + j] = (unsigned char)c;
      back = __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3)));
    } else {
      const __nv_bfloat16 c = __float2bfloat16_rn(v);
      ((__nv_bfloat16 *)out)[q * len + j] = c;
      back = __bfloat162float(c);
    }
    if (j < d_s) {
      const float r = fmaf(-s, back, src[j]);
      r2 = fmaf(r, r, r2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if (lane == 0) qrho[q] = sqrtf(r2);
}

// Qt[t][kb][r][0:128 B] = row pair_q[tile_beg[t] + r] of the low-precision
// queries at block kb (rpt rows per tile and block); rows past the tile's
// count are left as they are (the scan computes them but never reads their
// results).  One CTA per tile: a thread takes a (row, 16-byte chunk) and
// copies it for every K-block, up to eight loads in flight, with the row's
// query index read once; grid (max_tiles).
__global__ void gather_qtiles_kernel(const unsigned char *__restrict__ qlow, int nkb,
                                     const int32_t *__restrict__ tile_beg,
                                     const int32_t *__restrict__ tile_cnt,
                                     const int *__restrict__ ntiles,
                                     const int32_t *__restrict__ pair_q, int rpt,
                                     unsigned char *__restrict__ qt) {
  const int t = blockIdx.x;
  if (t >= *ntiles) return;
  const int beg = tile_beg[t], cnt = tile_cnt[t];
  for (int e = threadIdx.x; e < cnt * 8; e += blockDim.x) {
    const int r = e >> 3, c = e & 7;
    const uint4 *src = (const uint4 *)(qlow + (int64_t)pair_q[beg + r] * nkb * 128) + c;
    uint4 *dst = (uint4 *)(qt + ((int64_t)t * nkb * rpt + r) * 128) + c;
    for (int k0 = 0; k0 < nkb; k0 += 8) {
      uint4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < nkb) v[u] = src[(k0 + u) * 8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < nkb) dst[(int64_t)(k0 + u) * rpt * 8] = v[u];
    }
  }
}

// ---------------------------------------------------------------- candidate segments
// qtot[q] = sum over slots of the list size rounded up to 8
__global__ void cand_count_kernel(const uint64_t *__restrict__ ckeys, int64_t B, int nprobe,
                                  const int64_t *__restrict__ list_off,
                                  int64_t *__restrict__ qtot) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B) return;
  int64_t t = 0;
  for (int s = 0; s < nprobe; ++s) {
    const int l = probe_list(ckeys[q * nprobe + s]);
    if (l >= 0) t += (list_off[l + 1] - list_off[l] + 7) & ~7ll;
  }
  qtot[q] = t;
}

// Exclusive scan (int64) of rounds of 8,192 values: 1024 threads x 8
// consecutive values (serial per thread, shuffle scan per warp, one scan of the
// warp sums).  One CTA walks [first, last) from `carry0` (the sum before
// first); with part != NULL a CTA per round only writes its round's sum there.
__device__ __forceinline__ void scan64_rounds(const int64_t *__restrict__ in, int64_t first,
                                              int64_t last, int64_t carry0,
                                              int64_t *__restrict__ out,
                                              int64_t *__restrict__ total,
                                              int64_t *__restrict__ part) {
  __shared__ int64_t wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = last;
  int64_t carry = carry0;
  for (int64_t base = first; base < n; base += 8192) {
    const int64_t i0 = base + (int64_t)tid * 8;
    int64_t v[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = i0 + j < n ? in[i0 + j] : 0;
      sum += v[j];
    }
    int64_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int64_t w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int64_t ex = carry + (warp > 0 ? wsum[warp - 1] : 0) + inc - sum;
    if (!part) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (i0 + j < n) out[i0 + j] = ex;
        ex += v[j];
      }
    }
    carry += wsum[31];
    __syncthreads();  // wsum is rewritten by the next round
  }
  if (tid == 0 && part) *part = carry;
  if (tid == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(1024) scan64_kernel(const int64_t *__restrict__ in, int64_t n,
                                                      int64_t *__restrict__ out,
                                                      int64_t *__restrict__ total) {
  scan64_rounds(in, 0, n, 0, out, total, nullptr);
}

// multi-CTA form: CTA b sums round b (part[b]), then rescans it from the
// exclusive prefix of the round sums (partx[b])
__global__ void __launch_bounds__(1024) scan64_part_kernel(const int64_t *__restrict__ in,
                                                           int64_t n, int64_t *__restrict__ part) {
  const int64_t b0 = (int64_t)blockIdx.x * 8192;
  scan64_rounds(in, b0, min(n, b0 + 8192), 0, nullptr, nullptr, part + blockIdx.x);
}

__global__ void __launch_bounds__(1024) scan64_apply_kernel(const int64_t *__restrict__ in,
                                                            int64_t n,
                                                            const int64_t *__restrict__ partx,
                                                            int64_t *__restrict__ out) {
  const int64_t b0 = (int64_t)blockIdx.x * 8192;
  scan64_rounds(in, b0, min(n, b0 + 8192), partx[blockIdx.x], out, nullptr, nullptr);
}

__global__ void cand_base_kernel(const uint64_t *__restrict__ ckeys, int64_t B, int nprobe,
                                 const int64_t *__restrict__ list_off,
                                 const int64_t *__restrict__ qbase, int64_t *__restrict__ pbase) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B) return;
  int64_t t = qbase[q];
  for (int s = 0; s < nprobe; ++s) {
    const int l = probe_list(ckeys[q * nprobe + s]);
    pbase[q * nprobe + s] = t;
    if (l >= 0) t += (list_off[l + 1] - list_off[l] + 7) & ~7ll;
  }
}

// exclusive scan of n int64 values (one CTA); *total = their sum when non-null
int launch_scan64(const int64_t *in, int64_t n, int64_t *out, int64_t *total, cudaStream_t st) {
  if (n <= 0) return ADANNS_OK;
  const int64_t nb = (n + 8191) / 8192;
  if (nb <= 2 || nb > 8192) {  // one or two rounds (or very many): one CTA
    scan64_kernel<<<1, 1024, 0, st>>>(in, n, out, total);
    ADN_LAUNCH("scan64_kernel");
    return ADANNS_OK;
  }
  // a CTA per round: round sums, their scan (one CTA, at most one round), the rounds
  Scratch s(st);
  int64_t *part, *partx;
  int rc;
  if ((rc = s.get(&part, (size_t)nb)) || (rc = s.get(&partx, (size_t)nb))) return rc;
  scan64_part_kernel<<<(unsigned)nb, 1024, 0, st>>>(in, n, part);
  ADN_LAUNCH("scan64_part_kernel");
  scan64_kernel<<<1, 1024, 0, st>>>(part, nb, partx, total);
  ADN_LAUNCH("scan64_kernel");
  scan64_apply_kernel<<<(unsigned)nb, 1024, 0, st>>>(in, n, partx, out);
  ADN_LAUNCH("scan64_apply_kernel");
  return ADANNS_OK;
}

// per-query candidate segments: qtot, qbase (exclusive scan) and pbase
int launch_cand_segments(const uint64_t *ckeys, int64_t B, int nprobe, const int64_t *list_off,
                         int64_t *qtot, int64_t *qbase, int64_t *pbase, cudaStream_t st) {
  if (B <= 0) return ADANNS_OK;
  const unsigned g = (unsigned)((B + 255) / 256);
  cand_count_kernel<<<g, 256, 0, st>>>(ckeys, B, nprobe, list_off, qtot);
  ADN_LAUNCH("cand_count_kernel");
  int rc;
  if ((rc = launch_scan64(qtot, B, qbase, nullptr, st))) return rc;
  cand_base_kernel<<<g, 256, 0, st>>>(ckeys, B, nprobe, list_off, qbase, pbase);
  ADN_LAUNCH("cand_base_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- tensor-core scan launcher
int launch_mma_scan(const void *qtiles, int64_t qrows, const void *xlow, int64_t xrows,
                    const MmaScanArgs &a, cudaStream_t st);
// tiles of 128 members x MMA_NARROW_QT queries (few queries per probed list)
int launch_mma_narrow(const void *qtiles, int64_t qrows, const void *xlow, int64_t xrows,
                      const MmaScanArgs &a, cudaStream_t st);

// Certified shortlist pruning (exact: the result equals the unpruned rerank).
// A shortlisted candidate c is dropped before the exact rerank when its key
// exceeds the k-th smallest shortlist key by more than the query's delta,
// i.e. when even its smallest possible exact distance is above the largest
// possible exact distance of k other candidates.  For unit-norm prefixes,
// with r_x = x - s_x x~ and r_q = P(q) - s_q q~ the residuals of the stored
// and the query's low-precision values,
//   P(q).x - (s_q q~).(s_x x~) = P(q).r_x + r_q.x - r_q.r_x,
// so by Cauchy-Schwarz |d_exact - d_approx| <= E_q with
//   E_q = 2 (R + rho_q + R rho_q) (1 + 1e-3) + e_rest,
// R = max over the index of nu_x |r_x[0:d_s]| (recorded when the tier is
// built), rho_q = |r_q| (computed with the query's low-precision copy) and
// e_rest bounding the FP32 tensor-core accumulation (2 d_pad 2^-22), the FP32
// norm and scale terms and the FP32 rerank's own rounding (8 (d_s + 2) 2^-24),
// plus 1e-4.  Keys are round(16384 d_approx) (+-2^-15), so c can be dropped
// when key_c > key_k + 2 * 16384 * (2^-15 + E_q).  Set ADANNS_OPT_RERANK_PRUNE = 0
// to rerank every shortlisted candidate.
static bool shortlist_prune_enabled() { return option(ADANNS_OPT_RERANK_PRUNE) != 0; }

static float shortlist_e_rest(int d_s, int d_pad) {
  return (float)(2.0 * d_pad * std::ldexp(1.0, -22) + 8.0 * (d_s + 2) * std::ldexp(1.0, -24) +
                 1e-4);
}

// Whether a search uses the filtered tensor-core scan (records carry a 16-bit
// member index, so every list must have at most 65,536 members).
static bool scan_filter_enabled(const adanns_index *idx) {
  return option(ADANNS_OPT_SCAN_FILTER) != 0 && idx->max_list <= 65536;
}

int search_mixed(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                 int nprobe, int k, int which, int kk, int64_t *out_ids, float *out_dist,
                 int32_t *out_probes, cudaStream_t st, const QueryBudgets *qb) {
  const int fp8 = which == 1;
  const int epb = fp8 ? 128 : 64;
  const int nkb = (d_s + epb - 1) / epb;
  const int nlist = idx->nlist;
  const int dcp = pad16(d_c), dsp = pad16(d_s);
  const bool filt = scan_filter_enabled(idx);
  // few queries per probed list: tiles of 128 members x 32 queries, where they
  // were measured faster than the wide tiles (16 K-blocks or more: d_s >= 1024
  // for BF16, 2048 for FP8), or at any d_s when the option asks for them
  // (with the default rule, a tile shape the autotuner recorded for this
  // bucket takes precedence)
  const int64_t nopt = option(ADANNS_OPT_NARROW_SCAN);
  const double qpl = (double)B * nprobe / nlist;
  const int tuned = nopt == 1 ? tuned_lowp_qt(which, d_s, qpl) : 0;
  const bool narrow = !filt && nopt != 0 &&
                      (tuned ? tuned == MMA_NARROW_QT
                             : qpl <= 24.0 && (nopt == 2 || nkb >= 16));
  const int qt = narrow ? MMA_NARROW_QT : 128;
  const int64_t seg_q = (int64_t)nprobe * (((int64_t)idx->max_list + 7) & ~7ll);
  // filtered: the keys of each query's nearest list, one segment per query
  const int64_t stride0 = ((int64_t)idx->max_list + 7) & ~7ll;
  const int64_t per_q = (filt ? seg_q * 4 + stride0 * 2 : seg_q * 2) +
                        (int64_t)nprobe * ((int64_t)nkb * 128 + 36) +
                        (int64_t)(dcp + dsp) * 4 + (int64_t)nkb * 128 + (int64_t)kk * 8 + 64;
  // slices bounded by a scratch budget (the candidate keys dominate it)
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, scratch_budget() / per_q));
  // work-item tiles: the filtered scan's two passes (slot 0; slots 1..) each
  // get their own, the unfiltered scan one set over every slot
  const int64_t tiles_a = filt ? (Bc + qt - 1) / qt + nlist : (Bc * nprobe + qt - 1) / qt + nlist;
  const int64_t tiles_b = filt && nprobe > 1 ? (Bc * (nprobe - 1) + qt - 1) / qt + nlist : 0;
  const int64_t max_tiles = tiles_a + tiles_b;
  const bool prune = shortlist_prune_enabled();
  const float rmax = idx->lowp_rmax[which][gran_index(d_s)] * 1.001f;
  const float e_rest = shortlist_e_rest(d_s, nkb * epb);
  Scratch s(st);
  float *qc, *qs, *qn2, *qsc, *qrho;
  uint64_t *ckeys;
  int32_t *lcnt, *lbeg, *lfill, *tbeg, *pair_q, *pair_out, *tl, *tb, *tc;
  int *ntiles, *counter, *rcnt = nullptr;
  int *err = idx->dev_err;
  int64_t *qtot, *qbase, *pbase, *cids;
  unsigned char *qlow, *qtile;
  uint16_t *cand = nullptr, *tau = nullptr, *cand0 = nullptr;
  uint32_t *rec = nullptr;
  int rc;
  if ((rc = s.get(&qc, (size_t)Bc * dcp)) || (rc = s.get(&qs, (size_t)Bc * dsp)) ||
      (rc = s.get(&qn2, Bc)) || (rc = s.get(&qsc, Bc)) || (rc = s.get(&qrho, Bc)) || (rc = s.get(&ckeys, (size_t)Bc * nprobe)) ||
      (rc = s.get(&lcnt, nlist)) || (rc = s.get(&lbeg, nlist)) || (rc = s.get(&lfill, nlist)) ||
      (rc = s.get(&tbeg, nlist)) || (rc = s.get(&pair_q, (size_t)Bc * nprobe)) ||
      (rc = s.get(&pair_out, (size_t)Bc * nprobe)) || (rc = s.get(&tl, max_tiles)) ||
      (rc = s.get(&tb, max_tiles)) || (rc = s.get(&tc, max_tiles)) || (rc = s.get(&ntiles, 2)) ||
      (rc = s.get(&counter, 3)) || (rc = s.get(&qtot, Bc)) ||
      (rc = s.get(&qbase, Bc)) || (rc = s.get(&pbase, (size_t)Bc * nprobe)) ||
      (rc = s.get(&cids, (size_t)Bc * kk)) || (rc = s.get(&qlow, (size_t)Bc * nkb * 128)) ||
      (rc = s.get(&qtile, (size_t)max_tiles * nkb * qt * 128)))
    return rc;
  if (filt) {
    if ((rc = s.get(&rec, (size_t)Bc * seg_q)) || (rc = s.get(&rcnt, (size_t)Bc * nprobe)) ||
        (rc = s.get(&tau, Bc)) || (rc = s.get(&cand0, (size_t)(Bc * stride0))))
      return rc;
  } else if ((rc = s.get(&cand, (size_t)Bc * seg_q))) {
    return rc;
  }
  // survivors and slow-path queries of the selection, for adanns_profile_read_counters
  unsigned long long *stats = nullptr;
  if (profiling() && (rc = s.get(&stats, 2))) return rc;
  const int gi = gran_index(d_s);
  const float *mscale = idx->invn + (int64_t)gi * idx->N;
  const float *cx = idx->lowp_cx[which] + (int64_t)gi * idx->N;
  const int64_t xrows = idx->N * (int64_t)idx->lowp_blocks[which];
  // one tensor-core scan over a tile set (tile arrays at offset t0, the set's
  // pairs at offset p0 of pair_out, its own tile count and work counter)
  // (thr non-null: the filtered second pass; keys0: the first pass's keys of
  // each query's nearest list, one segment of stride0 per query)
  auto scan = [&](int64_t t0, int64_t ntile_cap, int64_t p0, int set, const uint16_t *thr,
                  uint16_t *keys0) -> int {
    MmaScanArgs m{};
    m.tile_list = tl + t0;
    m.tile_beg = tb + t0;
    m.tile_cnt = tc + t0;
    m.ntiles_dev = ntiles + set;
    m.list_off = idx->list_off;
    m.pair_out = pair_out + p0;
    m.pbase = pbase;
    m.cx = cx;
    m.qn2 = qn2;
    m.qsc = qsc;
    m.nprobe = nprobe;
    m.nkb = nkb;
    m.d_blocks = idx->lowp_blocks[which];
    m.cand = keys0 ? keys0 : cand;
    m.pstride = keys0 ? stride0 : 0;
    m.rec = thr ? rec : nullptr;
    m.rcnt = thr ? rcnt : nullptr;
    m.tau = thr;
    m.err = err;
    m.tile_counter = counter + 1 + set;  // zeroed with the cluster-mapping counter
    m.fp8 = fp8;
    m.few = (double)B * nprobe <= 24.0 * nlist ? 1 : 0;
    return narrow ? launch_mma_narrow(qtile + t0 * nkb * qt * 128, ntile_cap * nkb * qt,
                                      idx->lowp[which], xrows, m, st)
                  : launch_mma_scan(qtile + t0 * nkb * 128 * 128, ntile_cap * nkb * 128,
                                    idx->lowp[which], xrows, m, st);
  };
  for (int64_t b0 = 0; b0 < B; b0 += Bc) {
    const int64_t nb = std::min(Bc, B - b0);
    {
      StageTimer t(ST_PREP, st);
      if ((rc = launch_prep_queries(queries + b0 * idx->d, nb, idx->d, d_c, d_s, idx->metric, qc,
                                    dcp, qs, dsp, st)))
        return rc;
      prep_lowp_kernel<<<(unsigned)((nb + 7) / 8), 256, 0, st>>>(qs, dsp, nb, d_s, fp8, nkb, qlow,
                                                                 qn2, qsc, qrho);
      ADN_LAUNCH("prep_lowp_kernel");
    }
    ADN_CUDA(cudaMemsetAsync(counter, 0, 3 * sizeof(int), st));
    {
      StageTimer t(ST_COARSE, st);
      if ((rc = run_coarse(idx, qc, dcp, nb, d_c, nprobe, ckeys, counter, st))) return rc;
      if (qb && (rc = launch_mask_probes(ckeys, nb, nprobe, qb->at(b0).np, st))) return rc;
    }
    int32_t *probes = out_probes ? out_probes + b0 * nprobe : nullptr;
    {
      StageTimer t(ST_INVERT, st);
      // tile set 0: every slot (unfiltered) or slot 0 (filtered); tile set 1:
      // slots 1.. (filtered); pairs of set 1 follow those of set 0
      const int ns0 = filt ? 1 : nprobe;
      if ((rc = launch_invert_probe_slots(ckeys, nb, nprobe, 0, ns0, nlist, qt, lcnt, lbeg, lfill,
                                          tbeg, pair_q, pair_out, tl, tb, tc, ntiles, probes, st)))
        return rc;
      gather_qtiles_kernel<<<(unsigned)tiles_a, 256, 0, st>>>(qlow, nkb, tb, tc, ntiles, pair_q, qt,
                                                              qtile);
      ADN_LAUNCH("gather_qtiles_kernel");
      if (tiles_b > 0) {
        const int64_t o1 = nb;  // pairs of set 0
        if ((rc = launch_invert_probe_slots(ckeys, nb, nprobe, 1, nprobe - 1, nlist, qt, lcnt,
                                            lbeg, lfill, tbeg, pair_q + o1, pair_out + o1,
                                            tl + tiles_a, tb + tiles_a, tc + tiles_a, ntiles + 1,
                                            probes, st)))
          return rc;
        gather_qtiles_kernel<<<(unsigned)tiles_b, 256, 0, st>>>(
            qlow, nkb, tb + tiles_a, tc + tiles_a, ntiles + 1, pair_q + o1, qt,
            qtile + tiles_a * nkb * qt * 128);
        ADN_LAUNCH("gather_qtiles_kernel");
      }
      if ((rc = launch_cand_segments(ckeys, nb, nprobe, idx->list_off, qtot, qbase, pbase, st)))
        return rc;
    }
    {
      StageTimer t(ST_MMA, st);
      if (filt) {
        // pass 1: every query's nearest list, every key written; its kk-th key
        // bounds the query's shortlist; pass 2: the other lists, filtered
        ADN_CUDA(cudaMemsetAsync(rcnt, 0, sizeof(int) * nb * nprobe, st));
        if ((rc = scan(0, tiles_a, 0, 0, nullptr, cand0))) return rc;
        if ((rc = launch_shortlist_tau(cand0, stride0, ckeys, idx->list_off, rec, rcnt, pbase,
                                       nprobe, kk, nb, tau, st)))
          return rc;
        if (tiles_b > 0 && (rc = scan(tiles_a, tiles_b, nb, 1, tau, nullptr))) return rc;
      } else if ((rc = scan(0, tiles_a, 0, 0, nullptr, nullptr))) {
        return rc;
      }
    }
    {
      StageTimer t(ST_SELECT, st);
      if (stats) ADN_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), st));
      rc = filt ? launch_select_surv(rec, rcnt, pbase, ckeys, nprobe, idx->list_off, kk, k, qrho,
                                     rmax, e_rest, prune ? 1 : 0, nb, cids, stats, st)
                : launch_select16(cand, ckeys, nprobe, qbase, idx->list_off, kk, k, qrho, rmax,
                                  e_rest, prune ? 1 : 0, nb, cids, stats, st);
      if (rc) return rc;
      if (stats) {
        profile_count(PC_SURVIVORS, (const int64_t *)stats, st);
        profile_count(PC_SELECT_SLOW, (const int64_t *)stats + 1, st);
      }
    }
    {
      StageTimer t(ST_RERANK, st);
      if ((rc = launch_rerank_lists(cids, kk, nb, qs, dsp, d_s, idx, mscale, k, out_ids + b0 * k,
                                    out_dist + b0 * k, st)))
        return rc;
      if (qb && (rc = launch_pad_rows(out_ids + b0 * k, out_dist + b0 * k, nb, k, qb->at(b0).k,
                                      st)))
        return rc;
    }
  }
  // a timed-out tensor-core pipeline sets the index's sticky status word,
  // reported (and cleared) by adanns_index_status
  return ADANNS_OK;
}

}  // namespace adn
