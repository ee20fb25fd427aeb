// C ABI: AdANNS-OPQ training / import and AdANNS-IVFOPQ search.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace adn {

int launch_gemm_f32(bool transA, int M, int N, int K, float alpha, const float *A, int lda,
                    const float *B, int ldb, float beta, float *C, int ldc, cudaStream_t st);
int launch_pq_assign(const float *z, int64_t n, int ldz, int M, int dsub, const float *C,
                     uint8_t *codes, float *mind, cudaStream_t st);
int launch_pq_update(const float *z, int64_t n, int ldz, int M, int dsub, const uint8_t *codes,
                     double *sums, int32_t *counts, float *C, cudaStream_t st);
int launch_pq_decode(const uint8_t *codes, int64_t n, int M, int dsub, const float *C, float *out,
                     int ldo, cudaStream_t st);
int launch_pq_lut(const float *z, int64_t B, int ldz, int M, int dsub, const float *C, float *lut,
                  cudaStream_t st);
int launch_sum_f32(const float *v, int64_t n, double *out, cudaStream_t st);
int launch_sum_sq(const float *v, int64_t n, double *out, cudaStream_t st);
int launch_permute_codes(const uint8_t *by_id, const int32_t *list_ids, int64_t N, int M,
                         uint8_t *lo, cudaStream_t st);
int launch_identity(float *R, int d, cudaStream_t st);
int polar_factor(const float *Mx, int d, float *R, cudaStream_t st);
int adc_query_tile(int M, int k);
int launch_list_mean(const adanns_index *x, int d_s, float *lcent, cudaStream_t st);
int launch_sub_list_centre(float *rows, int64_t n, int ldr, int d_s, const int64_t *ids64,
                           const int32_t *ids32, const int32_t *assign, const float *lcent,
                           cudaStream_t st);
int launch_residual_tables(const float *w, int nlist, int d_s, int M, const float *C, float *S,
                           float *w2, cudaStream_t st);
struct AdcArgs;
int launch_rerank(const int64_t *cand, int kr, int64_t B, const float *qs, int ldq, int d_s,
                  const adanns_index *idx, const float *mscale, int k, int64_t *out_ids,
                  float *out_dist, cudaStream_t st);
int launch_adc(const uint8_t *codes, const int64_t *list_off, const int32_t *list_ids, int M,
               const float *lut, const int32_t *tl, const int32_t *tb, const int32_t *tc,
               const int *ntiles, int *counter, const int32_t *pair_q, const int32_t *pair_out,
               int k, uint64_t *out_keys, int qa, cudaStream_t st);

namespace {

cudaStream_t S(void *p) { return (cudaStream_t)p; }

// The ADC stage writes every probed member's distance and selects the top k'
// per query afterwards (adc_dist_kernel + select32_kernel) when n_p <= 256;
// ADANNS_OPT_ADC_SELECT = 0 keeps a running top-k' per (query, list) instead
// (adc_scan_kernel + merge).
bool adc_select_enabled(int nprobe) {
  return nprobe <= 256 && option(ADANNS_OPT_ADC_SELECT) != 0;
}


uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

std::vector<int64_t> seeded_sample(uint64_t seed, int64_t n, int64_t take) {
  std::vector<int64_t> a((size_t)n);
  for (int64_t i = 0; i < n; ++i) a[(size_t)i] = i;
  uint64_t st = seed;
  for (int64_t i = 0; i < take; ++i) {
    const int64_t j = i + (int64_t)(splitmix64(st) % (uint64_t)(n - i));
    std::swap(a[(size_t)i], a[(size_t)j]);
  }
  a.resize((size_t)take);
  return a;
}

__global__ void init_codebooks_kernel(const float *__restrict__ z, int ldz, const int64_t *rows,
                                      int M, int dsub, float *__restrict__ C) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * 256 * dsub) return;
  const int m = (int)(e / (256 * dsub));
  const int c = (int)((e / dsub) % 256);
  const int t = (int)(e % dsub);
  C[e] = z[rows[c] * ldz + (int64_t)m * dsub + t];
}

__global__ void widen_ids_kernel(const int32_t *__restrict__ a, int64_t n, int64_t *__restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

__global__ void sub_kernel(float *__restrict__ a, const float *__restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] -= b[i];
}

int check_opq_shape(int d_s, int M, int d) {
  if (gran_index(d_s) < 0 || d_s > d)
    return fail(ADANNS_ERR_DIM, "d_s = " + std::to_string(d_s) +
                                    " is not an MR granularity within the stored dimension");
  if (M < 1 || d_s % M != 0) return fail(ADANNS_ERR_ARG, "M must divide d_s");
  if (d_s / M > 64) return fail(ADANNS_ERR_ARG, "sub-vectors above 64 dimensions");
  return ADANNS_OK;
}

int read_double(const double *dev, double *host, cudaStream_t st) {
  ADN_CUDA(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  ADN_CUDA(cudaStreamSynchronize(st));
  return ADANNS_OK;
}

// Lloyd steps of every subspace on z (n x d_s): assign, update; then a final
// assignment.  Returns the distortion (mean squared reconstruction error).
int pq_lloyd(const float *z, int64_t n, int d_s, int M, int iters, float *C, uint8_t *codes,
             float *mind, double *sums, int32_t *counts, double *acc, double *distortion,
             cudaStream_t st) {
  const int dsub = d_s / M;
  int rc;
  for (int it = 0; it < iters; ++it) {
    if ((rc = launch_pq_assign(z, n, d_s, M, dsub, C, codes, nullptr, st))) return rc;
    if ((rc = launch_pq_update(z, n, d_s, M, dsub, codes, sums, counts, C, st))) return rc;
  }
  if ((rc = launch_pq_assign(z, n, d_s, M, dsub, C, codes, mind, st))) return rc;
  if ((rc = launch_sum_f32(mind, n * M, acc, st))) return rc;
  double tot = 0.0;
  if ((rc = read_double(acc, &tot, st))) return rc;
  *distortion = tot / (double)n;
  return ADANNS_OK;
}

void free_residual(adanns_index *x) {
  cudaFree(x->opq_lcent);
  cudaFree(x->opq_w);
  cudaFree(x->opq_w2);
  cudaFree(x->opq_S);
  x->opq_lcent = x->opq_w = x->opq_w2 = x->opq_S = nullptr;
}

void free_opq(adanns_index *x) {
  cudaFree(x->opq_R);
  cudaFree(x->opq_C);
  cudaFree(x->codes);
  x->opq_R = x->opq_C = nullptr;
  x->codes = nullptr;
  x->opq_ds = x->opq_M = 0;
  free_residual(x);
}

int alloc_residual(adanns_index *x, int d_s, int M) {
  const size_t nl = (size_t)x->nlist;
  if (cudaMalloc(&x->opq_lcent, sizeof(float) * nl * d_s) != cudaSuccess ||
      cudaMalloc(&x->opq_w, sizeof(float) * nl * d_s) != cudaSuccess ||
      cudaMalloc(&x->opq_w2, sizeof(float) * nl) != cudaSuccess ||
      cudaMalloc(&x->opq_S, sizeof(float) * nl * M * 256) != cudaSuccess) {
    cudaGetLastError();
    free_residual(x);
    return fail(ADANNS_ERR_OOM, "residual table allocation failed");
  }
  return ADANNS_OK;
}

// w = lcent R, |w_l|^2 and the per-list tables S from the index's R and codebooks
int finish_residual(adanns_index *x, cudaStream_t st) {
  const int d_s = x->opq_ds, M = x->opq_M;
  int rc;
  if ((rc = launch_gemm_f32(false, x->nlist, d_s, d_s, 1.f, x->opq_lcent, d_s, x->opq_R, d_s, 0.f,
                            x->opq_w, d_s, st)))
    return rc;
  return launch_residual_tables(x->opq_w, x->nlist, d_s, M, x->opq_C, x->opq_S, x->opq_w2, st);
}

int alloc_opq(adanns_index *x, int d_s, int M) {
  free_opq(x);
  const int dsub = d_s / M;
  if (cudaMalloc(&x->opq_R, sizeof(float) * d_s * d_s) != cudaSuccess ||
      cudaMalloc(&x->opq_C, sizeof(float) * M * 256 * dsub) != cudaSuccess ||
      cudaMalloc(&x->codes, (size_t)x->N * M) != cudaSuccess) {
    cudaGetLastError();
    free_opq(x);
    return fail(ADANNS_ERR_OOM, "OPQ allocation failed");
  }
  x->opq_ds = d_s;
  x->opq_M = M;
  return ADANNS_OK;
}

// codes of all N database vectors in list order: z = P_ds(x) R, nearest codewords
int encode_lists(adanns_index *x, const float *db, cudaStream_t st) {
  const int d_s = x->opq_ds, M = x->opq_M, dsp = pad16(d_s);
  const int64_t rows = std::min<int64_t>(x->N, 1 << 18);
  Scratch s(st);
  int64_t *r64;
  float *xn, *z;
  int rc;
  if ((rc = s.get(&r64, rows)) || (rc = s.get(&xn, (size_t)rows * dsp)) ||
      (rc = s.get(&z, (size_t)rows * d_s)))
    return rc;
  for (int64_t p0 = 0; p0 < x->N; p0 += rows) {
    const int64_t n = std::min(rows, x->N - p0);
    widen_ids_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x->list_ids + p0, n, r64);
    ADN_LAUNCH("widen_ids_kernel");
    if ((rc = launch_gather_normalize(db, n, x->d, r64, d_s, x->metric, xn, dsp, st))) return rc;
    if (x->opq_lcent &&
        (rc = launch_sub_list_centre(xn, n, dsp, d_s, r64, nullptr, x->assign, x->opq_lcent, st)))
      return rc;
    if ((rc = launch_gemm_f32(false, (int)n, d_s, d_s, 1.f, xn, dsp, x->opq_R, d_s, 0.f, z, d_s,
                              st)))
      return rc;
    if ((rc = launch_pq_assign(z, n, d_s, M, d_s / M, x->opq_C, x->codes + p0 * M, nullptr, st)))
      return rc;
  }
  return ADANNS_OK;
}

// AdANNS-IVFOPQ search with the distance-then-select ADC stage (Sec. 4.3):
// per chunk of queries, prep -> cluster mapping -> (list, query tile) work
// items -> LUTs -> every probed member's ADC distance into the query's
// candidate segment -> the k' smallest (distance, id) per query -> the k best
// (no rerank) or the exact FP32 rerank of the k'.
// qb (or null): per-query nprobe and k, at most the call's nprobe and k (rows
// of k entries, a query's own k results first, then padding)
int search_ivfopq_select(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                         int nprobe, int k, int kr, bool rerank, int64_t *out_ids, float *out_dist,
                         int32_t *out_probes, cudaStream_t st, const QueryBudgets *qb = nullptr) {
  const int d_s = idx->opq_ds, M = idx->opq_M, dsub = d_s / M;
  const int nlist = idx->nlist;
  const int dcp = pad16(d_c), dsp = pad16(d_s);
  const int qa = adc_dist_query_tile(M);
  const int64_t seg_q = max_probe_members(idx, nprobe);
  const int64_t per_q = seg_q * 4 + (int64_t)(dcp + dsp + d_s) * 4 + (int64_t)M * 1024 +
                        (int64_t)kr * 16 + (int64_t)nprobe * 40 + 16;
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, scratch_budget() / per_q));
  const int64_t max_tiles = (Bc * nprobe + qa - 1) / qa + nlist;
  Scratch s(st);
  float *qc, *qs, *z, *lut;
  uint64_t *ckeys, *keys;
  uint32_t *cand;
  int64_t *qtot, *qbase, *pbase, *cids;
  int32_t *lcnt, *lbeg, *lfill, *tbeg, *pair_q, *pair_out, *tl, *tb, *tc;
  int *ntiles, *counter;
  int rc;
  if ((rc = s.get(&qc, (size_t)Bc * dcp)) || (rc = s.get(&qs, (size_t)Bc * dsp)) ||
      (rc = s.get(&z, (size_t)Bc * d_s)) || (rc = s.get(&lut, (size_t)Bc * M * 256)) ||
      (rc = s.get(&ckeys, (size_t)Bc * nprobe)) || (rc = s.get(&cand, (size_t)(Bc * seg_q))) ||
      (rc = s.get(&keys, (size_t)Bc * kr)) || (rc = s.get(&cids, (size_t)Bc * kr)) ||
      (rc = s.get(&qtot, (size_t)Bc)) || (rc = s.get(&qbase, (size_t)Bc)) ||
      (rc = s.get(&pbase, (size_t)Bc * nprobe)) || (rc = s.get(&lcnt, nlist)) ||
      (rc = s.get(&lbeg, nlist)) || (rc = s.get(&lfill, nlist)) || (rc = s.get(&tbeg, nlist)) ||
      (rc = s.get(&pair_q, (size_t)Bc * nprobe)) || (rc = s.get(&pair_out, (size_t)Bc * nprobe)) ||
      (rc = s.get(&tl, max_tiles)) || (rc = s.get(&tb, max_tiles)) ||
      (rc = s.get(&tc, max_tiles)) || (rc = s.get(&ntiles, 1)) || (rc = s.get(&counter, 2)))
    return rc;
  const float *mscale = idx->metric == ADANNS_METRIC_L2_PREFIXNORM
                            ? idx->invn + (int64_t)gran_index(d_s) * idx->N
                            : nullptr;
  for (int64_t b0 = 0; b0 < B; b0 += Bc) {
    const int64_t nb = std::min(Bc, B - b0);
    {
      StageTimer t(ST_PREP, st);
      if ((rc = launch_prep_queries(queries + b0 * idx->d, nb, idx->d, d_c, d_s, idx->metric, qc,
                                    dcp, qs, dsp, st)))
        return rc;
    }
    ADN_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st));
    {
      StageTimer t(ST_COARSE, st);
      if ((rc = run_coarse(idx, qc, dcp, nb, d_c, nprobe, ckeys, counter, st))) return rc;
      if (qb && (rc = launch_mask_probes(ckeys, nb, nprobe, qb->at(b0).np, st))) return rc;
    }
    {
      StageTimer t(ST_INVERT, st);
      if ((rc = launch_invert_probes(ckeys, nb, nprobe, nlist, qa, lcnt, lbeg, lfill, tbeg, pair_q,
                                     pair_out, tl, tb, tc, ntiles,
                                     out_probes ? out_probes + b0 * nprobe : nullptr, st)))
        return rc;
      if ((rc = launch_cand_segments(ckeys, nb, nprobe, idx->list_off, qtot, qbase, pbase, st)))
        return rc;
    }
    {
      StageTimer t(ST_LUT, st);
      if ((rc = launch_gemm_f32(false, (int)nb, d_s, d_s, 1.f, qs, dsp, idx->opq_R, d_s, 0.f, z,
                                d_s, st)))
        return rc;
      if ((rc = launch_pq_lut(z, nb, d_s, M, dsub, idx->opq_C, lut, st))) return rc;
    }
    {
      StageTimer t(ST_ADC, st);
      // few work items (few queries, or one long list as in the exhaustive
      // search): split each list into member ranges so every SM has work
      const int64_t tiles_est = (nb * nprobe + qa - 1) / qa;
      const int64_t target = (int64_t)num_sms() * 4;
      const int nsplit = tiles_est >= target
                             ? 1
                             : (int)std::min<int64_t>((target + tiles_est - 1) / tiles_est,
                                                      ((int64_t)idx->max_list + 255) / 256);
      if ((rc = launch_adc_dist(idx->codes, idx->list_off, M, lut, tl, tb, tc, ntiles, counter + 1,
                                pair_q, pair_out, pbase, cand, qa, nsplit, st, idx->opq_S,
                                idx->opq_w, idx->opq_w2, z, d_s)))
        return rc;
    }
    {
      StageTimer t(ST_MERGE, st);
      if ((rc = launch_select32(cand, ckeys, nprobe, qbase, idx->list_off, idx->list_ids, nb, kr,
                                keys, st)))
        return rc;
      if (!rerank &&
          (rc = launch_final_topk(keys, kr, nb, k, out_ids + b0 * k, out_dist + b0 * k, st)))
        return rc;
    }
    if (rerank) {
      StageTimer t(ST_RERANK, st);
      if ((rc = launch_keys_to_ids(keys, nb * kr, cids, st))) return rc;
      if ((rc = launch_rerank(cids, kr, nb, qs, dsp, d_s, idx, mscale, k, out_ids + b0 * k,
                              out_dist + b0 * k, st)))
        return rc;
    }
    if (qb && (rc = launch_pad_rows(out_ids + b0 * k, out_dist + b0 * k, nb, k, qb->at(b0).k, st)))
      return rc;
  }
  return ADANNS_OK;
}

}  // namespace
}  // namespace adn

using namespace adn;

extern "C" {

int adanns_opq_encode(const float *x, int64_t n, int ld, int d_s, int M, int metric,
                      const float *R, const float *codebooks, uint8_t *codes, void *cuda_stream) {
  if (!x || !R || !codebooks || !codes) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (n < 0 || ld < d_s) return fail(ADANNS_ERR_ARG, "bad sizes");
  int rc;
  if ((rc = check_opq_shape(d_s, M, ld))) return rc;
  if (metric != ADANNS_METRIC_L2 && metric != ADANNS_METRIC_L2_PREFIXNORM)
    return fail(ADANNS_ERR_ARG, "unknown metric");
  if (n == 0) return ADANNS_OK;
  cudaStream_t st = S(cuda_stream);
  const int dsp = pad16(d_s);
  const int64_t rows = std::min<int64_t>(n, 1 << 18);
  Scratch s(st);
  float *xn, *z;
  if ((rc = s.get(&xn, (size_t)rows * dsp)) || (rc = s.get(&z, (size_t)rows * d_s))) return rc;
  for (int64_t i0 = 0; i0 < n; i0 += rows) {
    const int64_t m = std::min(rows, n - i0);
    if ((rc = launch_gather_normalize(x + i0 * ld, m, ld, nullptr, d_s, metric, xn, dsp, st)))
      return rc;
    if ((rc = launch_gemm_f32(false, (int)m, d_s, d_s, 1.f, xn, dsp, R, d_s, 0.f, z, d_s, st)))
      return rc;
    if ((rc = launch_pq_assign(z, m, d_s, M, d_s / M, codebooks, codes + i0 * M, nullptr, st)))
      return rc;
  }
  return ADANNS_OK;
}

int adanns_pq_update(const float *z, int64_t n, int d_s, int M, const uint8_t *codes,
                     float *codebooks, void *cuda_stream) {
  if (!z || !codes || !codebooks) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (n < 0 || M < 1 || d_s % M != 0) return fail(ADANNS_ERR_ARG, "bad sizes");
  cudaStream_t st = S(cuda_stream);
  const int dsub = d_s / M;
  Scratch s(st);
  double *sums;
  int32_t *counts;
  int rc;
  if ((rc = s.get(&sums, (size_t)M * 256 * dsub)) || (rc = s.get(&counts, (size_t)M * 256)))
    return rc;
  return launch_pq_update(z, n, d_s, M, dsub, codes, sums, counts, codebooks, st);
}

int adanns_procrustes(const float *Y, const float *Zhat, int64_t n, int d_s, float *R,
                      void *cuda_stream) {
  if (!Y || !Zhat || !R) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (n < 1 || n > INT32_MAX || d_s < 1) return fail(ADANNS_ERR_ARG, "bad sizes");
  cudaStream_t st = S(cuda_stream);
  Scratch s(st);
  float *Mx;
  int rc;
  if ((rc = s.get(&Mx, (size_t)d_s * d_s))) return rc;
  if ((rc = launch_gemm_f32(true, d_s, d_s, (int)n, 1.f, Y, d_s, Zhat, d_s, 0.f, Mx, d_s, st)))
    return rc;
  return polar_factor(Mx, d_s, R, st);
}

static int build_opq_impl(adanns_index *idx, const float *db, int d_s, int M, int opq_iters,
                          int pq_iters, int final_iters, int64_t train_n, uint64_t seed,
                          double *trace, bool residual, void *cuda_stream);

int adanns_build_opq(adanns_index *idx, const float *db, int d_s, int M, int opq_iters,
                     int pq_iters, int final_iters, int64_t train_n, uint64_t seed, double *trace,
                     void *cuda_stream) {
  return build_opq_impl(idx, db, d_s, M, opq_iters, pq_iters, final_iters, train_n, seed, trace,
                        false, cuda_stream);
}

int adanns_build_opq_residual(adanns_index *idx, const float *db, int d_s, int M, int opq_iters,
                              int pq_iters, int final_iters, int64_t train_n, uint64_t seed,
                              double *trace, void *cuda_stream) {
  return build_opq_impl(idx, db, d_s, M, opq_iters, pq_iters, final_iters, train_n, seed, trace,
                        true, cuda_stream);
}

static int build_opq_impl(adanns_index *idx, const float *db, int d_s, int M, int opq_iters,
                          int pq_iters, int final_iters, int64_t train_n, uint64_t seed,
                          double *trace, bool residual, void *cuda_stream) {
  if (!idx || !db) return fail(ADANNS_ERR_ARG, "NULL argument");
  int rc;
  if ((rc = check_opq_shape(d_s, M, idx->d))) return rc;
  if (opq_iters < 0 || pq_iters < 0 || final_iters < 0 || train_n < 1 || train_n > idx->N ||
      train_n > INT32_MAX)
    return fail(ADANNS_ERR_ARG, "bad OPQ schedule or training size");
  cudaStream_t st = S(cuda_stream);
  const int dsub = d_s / M;
  const int64_t n = train_n;
  std::vector<int64_t> S1 = seeded_sample(seed + 2, idx->N, n);
  std::vector<int64_t> P = seeded_sample(seed + 3, n, std::min<int64_t>(256, n));
  std::vector<int64_t> init(256);
  for (int c = 0; c < 256; ++c) init[c] = P[(size_t)(c % (int64_t)P.size())];
  if ((rc = alloc_opq(idx, d_s, M))) return rc;
  if (residual) {
    if ((rc = alloc_residual(idx, d_s, M)) || (rc = launch_list_mean(idx, d_s, idx->opq_lcent, st))) {
      free_opq(idx);
      return rc;
    }
  }
  Scratch s(st);
  int64_t *d_s1, *d_init;
  float *Y, *Z, *Zh, *Mx, *mind;
  uint8_t *codes;
  double *sums, *acc;
  int32_t *counts;
  if ((rc = s.get(&d_s1, n)) || (rc = s.get(&d_init, 256)) ||
      (rc = s.get(&Y, (size_t)n * d_s)) || (rc = s.get(&Z, (size_t)n * d_s)) ||
      (rc = s.get(&Zh, (size_t)n * d_s)) || (rc = s.get(&Mx, (size_t)d_s * d_s)) ||
      (rc = s.get(&mind, (size_t)n * M)) || (rc = s.get(&codes, (size_t)n * M)) ||
      (rc = s.get(&sums, (size_t)M * 256 * dsub)) || (rc = s.get(&acc, 1)) ||
      (rc = s.get(&counts, (size_t)M * 256)))
    return rc;
  ADN_CUDA(cudaMemcpyAsync(d_s1, S1.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  ADN_CUDA(cudaMemcpyAsync(d_init, init.data(), sizeof(int64_t) * 256, cudaMemcpyHostToDevice, st));
  if ((rc = launch_gather_normalize(db, n, idx->d, d_s1, d_s, idx->metric, Y, d_s, st))) return rc;
  if (residual && (rc = launch_sub_list_centre(Y, n, d_s, d_s, d_s1, nullptr, idx->assign,
                                               idx->opq_lcent, st)))
    return rc;
  if ((rc = launch_identity(idx->opq_R, d_s, st))) return rc;
  int nt = 0;
  bool have_C = false;
  const int64_t nd = n * d_s;
  const unsigned gnd = (unsigned)((nd + 255) / 256);
  auto put = [&](double v) {
    if (trace) trace[nt] = v;
    ++nt;
  };
  for (int t = 0; t < opq_iters; ++t) {
    if ((rc = launch_gemm_f32(false, (int)n, d_s, d_s, 1.f, Y, d_s, idx->opq_R, d_s, 0.f, Z, d_s,
                              st)))
      return rc;
    double dist = 0.0;
    if (!have_C) {
      init_codebooks_kernel<<<(unsigned)((M * 256 * dsub + 255) / 256), 256, 0, st>>>(
          Z, d_s, d_init, M, dsub, idx->opq_C);
      ADN_LAUNCH("init_codebooks_kernel");
      have_C = true;
    } else {
      if ((rc = pq_lloyd(Z, n, d_s, M, 0, idx->opq_C, codes, mind, sums, counts, acc, &dist, st)))
        return rc;
      put(dist);
    }
    if ((rc = pq_lloyd(Z, n, d_s, M, pq_iters, idx->opq_C, codes, mind, sums, counts, acc, &dist,
                       st)))
      return rc;
    put(dist);
    if ((rc = launch_pq_decode(codes, n, M, dsub, idx->opq_C, Zh, d_s, st))) return rc;
    if ((rc = launch_gemm_f32(true, d_s, d_s, (int)n, 1.f, Y, d_s, Zh, d_s, 0.f, Mx, d_s, st)))
      return rc;
    if ((rc = polar_factor(Mx, d_s, idx->opq_R, st))) return rc;
    // ||Y R - Zhat||^2 / n after the rotation update
    if ((rc = launch_gemm_f32(false, (int)n, d_s, d_s, 1.f, Y, d_s, idx->opq_R, d_s, 0.f, Z, d_s,
                              st)))
      return rc;
    sub_kernel<<<gnd, 256, 0, st>>>(Z, Zh, nd);
    ADN_LAUNCH("sub_kernel");
    if ((rc = launch_sum_sq(Z, nd, acc, st))) return rc;
    double tot = 0.0;
    if ((rc = read_double(acc, &tot, st))) return rc;
    put(tot / (double)n);
  }
  if ((rc = launch_gemm_f32(false, (int)n, d_s, d_s, 1.f, Y, d_s, idx->opq_R, d_s, 0.f, Z, d_s,
                            st)))
    return rc;
  if (!have_C) {
    init_codebooks_kernel<<<(unsigned)((M * 256 * dsub + 255) / 256), 256, 0, st>>>(
        Z, d_s, d_init, M, dsub, idx->opq_C);
    ADN_LAUNCH("init_codebooks_kernel");
  }
  double dist = 0.0;
  if ((rc = pq_lloyd(Z, n, d_s, M, final_iters, idx->opq_C, codes, mind, sums, counts, acc, &dist,
                     st)))
    return rc;
  put(dist);
  if ((rc = encode_lists(idx, db, st))) return rc;
  if (residual && (rc = finish_residual(idx, st))) return rc;
  ADN_CUDA(cudaStreamSynchronize(st));
  return ADANNS_OK;
}

int adanns_index_set_opq(adanns_index *idx, int d_s, int M, const float *R,
                         const float *codebooks, const uint8_t *codes_by_id, void *cuda_stream) {
  if (!idx || !R || !codebooks || !codes_by_id) return fail(ADANNS_ERR_ARG, "NULL argument");
  int rc;
  if ((rc = check_opq_shape(d_s, M, idx->d))) return rc;
  cudaStream_t st = S(cuda_stream);
  if ((rc = alloc_opq(idx, d_s, M))) return rc;
  ADN_CUDA(cudaMemcpyAsync(idx->opq_R, R, sizeof(float) * d_s * d_s, cudaMemcpyDeviceToDevice, st));
  ADN_CUDA(cudaMemcpyAsync(idx->opq_C, codebooks, sizeof(float) * M * 256 * (d_s / M),
                           cudaMemcpyDeviceToDevice, st));
  if ((rc = launch_permute_codes(codes_by_id, idx->list_ids, idx->N, M, idx->codes, st))) return rc;
  ADN_CUDA(cudaStreamSynchronize(st));
  return ADANNS_OK;
}

int adanns_index_set_opq_residual(adanns_index *idx, int d_s, int M, const float *R,
                                  const float *codebooks, const uint8_t *codes_by_id,
                                  const float *list_centres, void *cuda_stream) {
  if (!list_centres) return fail(ADANNS_ERR_ARG, "NULL argument");
  int rc;
  if ((rc = adanns_index_set_opq(idx, d_s, M, R, codebooks, codes_by_id, cuda_stream))) return rc;
  cudaStream_t st = S(cuda_stream);
  if ((rc = alloc_residual(idx, d_s, M))) return rc;
  ADN_CUDA(cudaMemcpyAsync(idx->opq_lcent, list_centres, sizeof(float) * idx->nlist * d_s,
                           cudaMemcpyDeviceToDevice, st));
  if ((rc = finish_residual(idx, st))) return rc;
  ADN_CUDA(cudaStreamSynchronize(st));
  return ADANNS_OK;
}

int adanns_index_get_list_centres(const adanns_index *idx, float *list_centres,
                                  void *cuda_stream) {
  if (!idx || !list_centres) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (!idx->opq_lcent) return fail(ADANNS_ERR_STATE, "the index has no residual OPQ codes");
  ADN_CUDA(cudaMemcpyAsync(list_centres, idx->opq_lcent, sizeof(float) * idx->nlist * idx->opq_ds,
                           cudaMemcpyDeviceToDevice, S(cuda_stream)));
  return ADANNS_OK;
}

int adanns_index_opq_info(const adanns_index *idx, int *d_s, int *M) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (d_s) *d_s = idx->codes ? idx->opq_ds : 0;
  if (M) *M = idx->codes ? idx->opq_M : 0;
  return ADANNS_OK;
}

int adanns_index_get_opq(const adanns_index *idx, float *R, float *codebooks,
                         uint8_t *codes_list_order, void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (!idx->codes) return fail(ADANNS_ERR_STATE, "the index has no OPQ data");
  cudaStream_t st = S(cuda_stream);
  const int d_s = idx->opq_ds, M = idx->opq_M;
  if (R) ADN_CUDA(cudaMemcpyAsync(R, idx->opq_R, sizeof(float) * d_s * d_s, cudaMemcpyDeviceToDevice, st));
  if (codebooks)
    ADN_CUDA(cudaMemcpyAsync(codebooks, idx->opq_C, sizeof(float) * M * 256 * (d_s / M),
                             cudaMemcpyDeviceToDevice, st));
  if (codes_list_order)
    ADN_CUDA(cudaMemcpyAsync(codes_list_order, idx->codes, (size_t)idx->N * M,
                             cudaMemcpyDeviceToDevice, st));
  return ADANNS_OK;
}

int adanns_search_ivfopq(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                         int nprobe, int k, int rerank_k, int64_t *out_ids, float *out_dist,
                         int32_t *out_probes, void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (!idx->codes) return fail(ADANNS_ERR_STATE, "the index has no OPQ data");
  if (B < 0 || B > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad batch size");
  if (B > 0 && (!queries || !out_ids || !out_dist)) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (gran_index(d_c) < 0 || d_c > idx->d_c)
    return fail(ADANNS_ERR_DIM, "d_c must be an MR granularity <= the index's clustering prefix " +
                                    std::to_string(idx->d_c));
  if (nprobe < 1 || nprobe > idx->nlist) return fail(ADANNS_ERR_ARG, "need 1 <= nprobe <= nlist");
  if (k < 1 || k > 1024) return fail(ADANNS_ERR_ARG, "need 1 <= k <= 1024");
  if (rerank_k != 0 && (rerank_k < k || rerank_k > 2048))
    return fail(ADANNS_ERR_ARG, "need rerank_k = 0 or k <= rerank_k <= 2048");
  if (B == 0) return ADANNS_OK;
  cudaStream_t st = S(cuda_stream);
  const int d_s = idx->opq_ds, M = idx->opq_M, dsub = d_s / M;
  const int nlist = idx->nlist;
  const int dcp = pad16(d_c), dsp = pad16(d_s);
  const int kr = rerank_k > 0 ? rerank_k : k;
  if (idx->opq_S && nprobe > 256)
    return fail(ADANNS_ERR_ARG, "residual IVF-OPQ search needs nprobe <= 256");
  if (adc_select_enabled(nprobe) || idx->opq_S)
    return search_ivfopq_select(idx, queries, B, d_c, nprobe, k, kr, rerank_k > 0, out_ids,
                                out_dist, out_probes, st);
  const int qa = adc_query_tile(M, kr);
  const int64_t per_q = (int64_t)nprobe * kr * 8 + (int64_t)(dcp + dsp + d_s) * 4 +
                        (int64_t)M * 1024 + (int64_t)kr * 12 + nprobe * 24;
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, (2ll << 30) / per_q));
  const int64_t max_tiles = (Bc * nprobe + qa - 1) / qa + nlist;
  Scratch s(st);
  float *qc, *qs, *z, *lut, *cdist;
  uint64_t *ckeys, *pkeys;
  int64_t *cids;
  int32_t *lcnt, *lbeg, *lfill, *tbeg, *pair_q, *pair_out, *tl, *tb, *tc;
  int *ntiles, *counter;
  int rc;
  if ((rc = s.get(&qc, (size_t)Bc * dcp)) || (rc = s.get(&qs, (size_t)Bc * dsp)) ||
      (rc = s.get(&z, (size_t)Bc * d_s)) || (rc = s.get(&lut, (size_t)Bc * M * 256)) ||
      (rc = s.get(&ckeys, (size_t)Bc * nprobe)) || (rc = s.get(&pkeys, (size_t)Bc * nprobe * kr)) ||
      (rc = s.get(&cids, (size_t)Bc * kr)) || (rc = s.get(&cdist, (size_t)Bc * kr)) ||
      (rc = s.get(&lcnt, nlist)) || (rc = s.get(&lbeg, nlist)) || (rc = s.get(&lfill, nlist)) ||
      (rc = s.get(&tbeg, nlist)) || (rc = s.get(&pair_q, (size_t)Bc * nprobe)) ||
      (rc = s.get(&pair_out, (size_t)Bc * nprobe)) || (rc = s.get(&tl, max_tiles)) ||
      (rc = s.get(&tb, max_tiles)) || (rc = s.get(&tc, max_tiles)) || (rc = s.get(&ntiles, 1)) ||
      (rc = s.get(&counter, 2)))
    return rc;
  const float *mscale = idx->metric == ADANNS_METRIC_L2_PREFIXNORM
                            ? idx->invn + (int64_t)gran_index(d_s) * idx->N
                            : nullptr;
  for (int64_t b0 = 0; b0 < B; b0 += Bc) {
    const int64_t nb = std::min(Bc, B - b0);
    {
      StageTimer t(ST_PREP, st);
      if ((rc = launch_prep_queries(queries + b0 * idx->d, nb, idx->d, d_c, d_s, idx->metric, qc,
                                    dcp, qs, dsp, st)))
        return rc;
    }
    ADN_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st));
    {
      StageTimer t(ST_COARSE, st);
      if ((rc = run_coarse(idx, qc, dcp, nb, d_c, nprobe, ckeys, counter, st))) return rc;
    }
    {
      StageTimer t(ST_INVERT, st);
      if ((rc = launch_invert_probes(ckeys, nb, nprobe, nlist, qa, lcnt, lbeg, lfill, tbeg, pair_q,
                                     pair_out, tl, tb, tc, ntiles,
                                     out_probes ? out_probes + b0 * nprobe : nullptr, st)))
        return rc;
    }
    {
      StageTimer t(ST_LUT, st);
      if ((rc = launch_gemm_f32(false, (int)nb, d_s, d_s, 1.f, qs, dsp, idx->opq_R, d_s, 0.f, z,
                                d_s, st)))
        return rc;
      if ((rc = launch_pq_lut(z, nb, d_s, M, dsub, idx->opq_C, lut, st))) return rc;
    }
    {
      StageTimer t(ST_ADC, st);
      if ((rc = launch_adc(idx->codes, idx->list_off, idx->list_ids, M, lut, tl, tb, tc, ntiles,
                           counter + 1, pair_q, pair_out, kr, pkeys, qa, st)))
        return rc;
    }
    if (rerank_k > 0) {
      {
        StageTimer t(ST_MERGE, st);
        if ((rc = launch_merge(pkeys, nb, nprobe, kr, cids, cdist, st))) return rc;
      }
      StageTimer t(ST_RERANK, st);
      if ((rc = launch_rerank(cids, kr, nb, qs, dsp, d_s, idx, mscale, k, out_ids + b0 * k,
                              out_dist + b0 * k, st)))
        return rc;
    } else {
      StageTimer t(ST_MERGE, st);
      if ((rc = launch_merge(pkeys, nb, nprobe, k, out_ids + b0 * k, out_dist + b0 * k, st)))
        return rc;
    }
  }
  return ADANNS_OK;
}

int adanns_search_ivfopq_budgets(const adanns_index *idx, const float *queries, int64_t B,
                                 int d_c, const int32_t *nprobe, const int32_t *k, int k_max,
                                 int rerank_k, int64_t *out_ids, float *out_dist,
                                 void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (!idx->codes) return fail(ADANNS_ERR_STATE, "the index has no OPQ data");
  if (B < 0 || B > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad batch size");
  if (B > 0 && (!queries || !out_ids || !out_dist || !nprobe || !k))
    return fail(ADANNS_ERR_ARG, "NULL argument");
  if (gran_index(d_c) < 0 || d_c > idx->d_c)
    return fail(ADANNS_ERR_DIM, "d_c must be an MR granularity <= the index's clustering prefix " +
                                    std::to_string(idx->d_c));
  if (k_max < 1 || k_max > 1024) return fail(ADANNS_ERR_ARG, "need 1 <= k_max <= 1024");
  if (rerank_k != 0 && (rerank_k < k_max || rerank_k > 2048))
    return fail(ADANNS_ERR_ARG, "need rerank_k = 0 or k_max <= rerank_k <= 2048");
  int np_max = 0;
  // staging array: nprobe, then k, of every query
  std::vector<int32_t> h((size_t)B * 2);
  for (int64_t i = 0; i < B; ++i) {
    const std::string at = " (query " + std::to_string(i) + ")";
    if (nprobe[i] < 1 || nprobe[i] > idx->nlist || nprobe[i] > 256)
      return fail(ADANNS_ERR_ARG, "need 1 <= nprobe <= min(nlist, 256)" + at);
    if (k[i] < 1 || k[i] > k_max) return fail(ADANNS_ERR_ARG, "need 1 <= k <= k_max" + at);
    np_max = std::max(np_max, (int)nprobe[i]);
    h[(size_t)i] = nprobe[i];
    h[(size_t)(B + i)] = k[i];
  }
  if (B == 0) return ADANNS_OK;
  cudaStream_t st = S(cuda_stream);
  Scratch s(st);
  int32_t *dq;
  int rc;
  if ((rc = s.get(&dq, h.size()))) return rc;
  // pageable source: staged by the copy call itself, so h may go when it returns
  ADN_CUDA(cudaMemcpyAsync(dq, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  QueryBudgets qb;
  qb.np = dq;
  qb.k = dq + B;
  const int kr = rerank_k > 0 ? rerank_k : k_max;
  return search_ivfopq_select(idx, queries, B, d_c, np_max, k_max, kr, rerank_k > 0, out_ids,
                              out_dist, nullptr, st, &qb);
}

}  // extern "C"
