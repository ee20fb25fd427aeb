// C ABI entry points: argument checks, scratch management and the launch
// sequence of each operation.  All arithmetic runs in the kernels.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace adn {
const char *last_error();

namespace {

cudaStream_t S(void *p) { return (cudaStream_t)p; }

// splitmix64 (Steele, Lea & Flood 2014) and a partial Fisher-Yates shuffle:
// the first `take` entries of a shuffle of [0, n), j = i + next() mod (n - i).
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

template <class T>
int dmalloc(T **p, size_t count) {
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ADANNS_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  return ADANNS_OK;
}

void free_index(adanns_index *x) {
  if (!x) return;
  cudaFree(x->centroids);
  cudaFree(x->cent_low);
  cudaFree(x->cent_sc);
  cudaFree(x->cent_n2);
  cudaFree(x->cent_pm);
  cudaFree(x->cent_off);
  cudaFree(x->list_off);
  cudaFree(x->list_ids);
  cudaFree(x->xpm);
  cudaFree(x->invn);
  cudaFree(x->dev_err);
  cudaFree(x->assign);
  cudaFree(x->pos_of_id);
  cudaFree(x->opq_R);
  cudaFree(x->opq_C);
  cudaFree(x->codes);
  for (int i = 0; i < 2; ++i) {
    cudaFree(x->lowp[i]);
    cudaFree(x->lowp_sx[i]);
    cudaFree(x->lowp_cx[i]);
  }
  for (int i = 0; i < 4; ++i) cudaFree(x->rr_cmap[i]);
  delete[] x->h_list_off;
  delete x;
}

int check_metric(int metric) {
  if (metric != ADANNS_METRIC_L2 && metric != ADANNS_METRIC_L2_PREFIXNORM)
    return fail(ADANNS_ERR_ARG, "unknown metric");
  return ADANNS_OK;
}

int check_gran(int m, int limit, const char *what) {
  if (gran_index(m) < 0)
    return fail(ADANNS_ERR_DIM, std::string(what) + " = " + std::to_string(m) +
                                    " is not an MR granularity (8,16,32,48,64,96,...,2048)");
  if (m > limit)
    return fail(ADANNS_ERR_DIM, std::string(what) + " = " + std::to_string(m) +
                                    " exceeds the available " + std::to_string(limit));
  return ADANNS_OK;
}

// prefix-major copy of an nc x dim centroid table as one list of nc members
int centroids_pm(const float *cent, int nc, int dim, float *out, cudaStream_t st) {
  return launch_prefix_major(cent, dim, dim, pad16(dim), nullptr, nullptr, nullptr, nc, out, st);
}

int scan_grid_default() { return 0; }

// top-1 sweep of `n` prepared points (rows of ldq) against a prefix-major
// centroid table; keys[i] = (distance, centroid)
int top1_sweep(const float *pts, int64_t n, int ldq, const float *cent_pm, const int64_t *cent_off,
               int nc, int dim, uint64_t *keys, int *counter, cudaStream_t st) {
  ScanArgs a{};
  a.xpm = cent_pm;
  a.d_pad = pad16(dim);
  a.dims = dim;
  a.list_off = cent_off;
  a.list_ids = nullptr;
  a.mscale = nullptr;
  a.qn = pts;
  a.ldq = ldq;
  a.nq = (int)n;
  a.counter = counter;
  a.k = 1;
  a.out_keys = keys;
  a.grid = scan_grid_default();
  (void)nc;
  ADN_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
  return launch_scan_f32(a, st);
}

// Nearest of nc centroids (nc x dim FP32 row-major `cent`, also prefix-major
// in cent_pm / cent_off) for n prepared points (rows of ldq floats):
// keys[i] = (distance bits << 32 | centroid), ties to the lower centroid.
// The Lloyd assignment step as a tensor-core GEMM: with at least 256
// centroids, dim <= 64 and the prefix-normalised metric, BF16 products of the
// points and a BF16 copy of the centroids (tcgen05) shortlist every centroid
// within the quantisation error bound of the best, and those are scored
// exactly in FP32 -- the cluster mapping's path with n_p = 1, so the result is
// the FP32 scan's.  Otherwise the FP32 scan.  err: the device status word of
// the tensor-core pipeline.
int nearest_centroid(const float *cent, int nc, int dim, int metric, const float *cent_pm,
                     const int64_t *cent_off, const float *pts, int64_t n, int ldq,
                     uint64_t *keys, int *counter, int *err, cudaStream_t st) {
  if (n <= 0) return ADANNS_OK;
  if (metric == ADANNS_METRIC_L2_PREFIXNORM && nc >= 256 && dim <= 64 &&
      option(ADANNS_OPT_COARSE_TC)) {
    adanns_index shell;
    shell.centroids = const_cast<float *>(cent);
    shell.nlist = nc;
    shell.d_c = dim;
    shell.dc_pad = pad16(dim);
    shell.metric = metric;
    shell.cent_pm = const_cast<float *>(cent_pm);
    shell.cent_off = const_cast<int64_t *>(cent_off);
    shell.dev_err = err;
    int rc = build_centroid_lowp(&shell, st);
    if (rc == ADANNS_OK) {
      // slices keep the 2-byte keys of (point, centroid) pairs near 1 GiB
      const int64_t rows = std::max<int64_t>(CT_SLICE_MIN, (1ll << 29) / ((nc + 7) & ~7));
      for (int64_t i0 = 0; i0 < n && rc == ADANNS_OK; i0 += rows)
        rc = launch_coarse_tc(&shell, pts + i0 * ldq, ldq, std::min(rows, n - i0), dim, 1,
                              keys + i0, st);
    }
    cudaStreamSynchronize(st);  // the table copies are released below
    cudaFree(shell.cent_low);
    cudaFree(shell.cent_sc);
    cudaFree(shell.cent_n2);
    if (rc != 1) return rc;  // 1: the shape does not fit the tensor-core path
  }
  return top1_sweep(pts, n, ldq, cent_pm, cent_off, nc, dim, keys, counter, st);
}

int make_cent_off(int64_t **off, int nc, cudaStream_t st) {
  int rc = dmalloc(off, 2);
  if (rc) return rc;
  int64_t h[2] = {0, (int64_t)nc};
  ADN_CUDA(cudaMemcpyAsync(*off, h, sizeof(h), cudaMemcpyHostToDevice, st));
  return ADANNS_OK;
}

constexpr int64_t SWEEP_ROWS = 1 << 20;  // points per assignment slice

// assign all N rows of db (first d_c coordinates, normalised per metric) to
// the nearest of nc centroids (row-major cent and its prefix-major table)
int assign_all(const float *db, int64_t N, int ld, int d_c, int metric, const float *cent,
               const float *cent_pm, const int64_t *cent_off, int nc, int32_t *assign,
               float *dist, int *err, cudaStream_t st) {
  Scratch s(st);
  const int dcp = pad16(d_c);
  const int64_t rows = std::min<int64_t>(N, SWEEP_ROWS);
  float *pn;
  uint64_t *keys;
  int *counter;
  int rc;
  if ((rc = s.get(&pn, (size_t)rows * dcp)) || (rc = s.get(&keys, (size_t)rows)) ||
      (rc = s.get(&counter, 1)))
    return rc;
  for (int64_t b0 = 0; b0 < N; b0 += rows) {
    const int64_t n = std::min(rows, N - b0);
    if ((rc = launch_gather_normalize(db + b0 * ld, n, ld, nullptr, d_c, metric, pn, dcp, st)))
      return rc;
    if ((rc = nearest_centroid(cent, nc, d_c, metric, cent_pm, cent_off, pn, n, dcp, keys, counter,
                               err, st)))
      return rc;
    if ((rc = launch_keys_to_result(keys, n, 1, nullptr, assign + b0, dist ? dist + b0 : nullptr,
                                    st)))
      return rc;
  }
  return ADANNS_OK;
}

int make_index(const float *db, int64_t N, int d, const float *centroids, int nlist, int d_c,
               const int32_t *assign, int metric, int storage, cudaStream_t st,
               adanns_index **out) {
  adanns_index *x = new adanns_index();
  x->N = N;
  x->d = d;
  x->d_pad = pad16(d);
  x->d_c = d_c;
  x->dc_pad = pad16(d_c);
  x->nlist = nlist;
  x->metric = metric;
  x->storage = storage;
  int rc;
  x->ng = 0;
  for (int g = 0; g < NGRAN; ++g)
    if (kGran[g] <= d) x->ng = g + 1;
  if ((rc = dmalloc(&x->centroids, (size_t)nlist * d_c)) ||
      (rc = dmalloc(&x->cent_pm, (size_t)nlist * x->dc_pad)) ||
      (rc = make_cent_off(&x->cent_off, nlist, st)) ||
      (rc = dmalloc(&x->list_off, (size_t)nlist + 1)) || (rc = dmalloc(&x->list_ids, (size_t)N)) ||
      (rc = dmalloc(&x->xpm, (size_t)N * x->d_pad)) ||
      (rc = dmalloc(&x->invn, (size_t)std::max(x->ng, 1) * N)) ||
      (rc = dmalloc(&x->assign, (size_t)N)) || (rc = dmalloc(&x->pos_of_id, (size_t)N)) ||
      (rc = dmalloc(&x->dev_err, 1))) {
    free_index(x);
    return rc;
  }
  auto bail = [&](int code) {
    cudaStreamSynchronize(st);
    free_index(x);
    return code;
  };
  if (cudaMemsetAsync(x->dev_err, 0, sizeof(int), st) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "clear status"));
  if (cudaMemcpyAsync(x->centroids, centroids, sizeof(float) * nlist * d_c,
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "copy centroids"));
  if ((rc = centroids_pm(x->centroids, nlist, d_c, x->cent_pm, st))) return bail(rc);
  if ((rc = build_centroid_lowp(x, st))) return bail(rc);
  if ((rc = build_csr(assign, N, nlist, x->list_off, x->list_ids, st))) return bail(rc);
  if ((rc = launch_prefix_major(db, d, d, x->d_pad, x->list_off, x->list_ids, assign, N, x->xpm,
                                st)))
    return bail(rc);
  if ((rc = launch_inv_norms(db, d, d, x->list_ids, N, metric, x->invn, x->ng, st)))
    return bail(rc);
  if (cudaMemcpyAsync(x->assign, assign, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "copy assignment"));
  if ((rc = launch_positions(x->list_ids, N, x->pos_of_id, st))) return bail(rc);
  if ((storage & ADANNS_STORE_BF16) && (rc = build_lowp(x, db, 0, st))) return bail(rc);
  if ((storage & ADANNS_STORE_FP8E4M3) && (rc = build_lowp(x, db, 1, st))) return bail(rc);
  x->h_list_off = new int64_t[nlist + 1];
  if (cudaMemcpyAsync(x->h_list_off, x->list_off, sizeof(int64_t) * (nlist + 1),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "copy list offsets"));
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bail(cuda_fail(e, "index build"));
  int64_t mx = 0;
  for (int l = 0; l < nlist; ++l) mx = std::max(mx, x->h_list_off[l + 1] - x->h_list_off[l]);
  x->max_list = (int)mx;
  if ((rc = build_rerank_order(x, st))) return bail(rc);
  *out = x;
  return ADANNS_OK;
}

}  // namespace

// Lists in a greedy nearest-neighbour chain of their centroids (start at list
// 0, then repeatedly the nearest list not yet taken; ties to the lower id), so
// lists next to each other in the order are probed by overlapping query sets.
// Above 4,096 lists the chain's quadratic cost is not paid: identity order.
int build_rerank_order(adanns_index *x, cudaStream_t st) {
  const int nl = x->nlist, dc = x->d_c;
  std::vector<int32_t> ord((size_t)nl);
  for (int i = 0; i < nl; ++i) ord[(size_t)i] = i;
  if (nl > 2 && nl <= 4096) {
    std::vector<float> c((size_t)nl * dc);
    ADN_CUDA(cudaMemcpyAsync(c.data(), x->centroids, sizeof(float) * c.size(),
                             cudaMemcpyDeviceToHost, st));
    ADN_CUDA(cudaStreamSynchronize(st));
    std::vector<char> used((size_t)nl, 0);
    int cur = 0;
    used[0] = 1;
    for (int i = 1; i < nl; ++i) {
      const float *a = c.data() + (size_t)cur * dc;
      int best = -1;
      double bd = 0.0;
      for (int j = 0; j < nl; ++j) {
        if (used[(size_t)j]) continue;
        const float *b = c.data() + (size_t)j * dc;
        double dd = 0.0;
        for (int t = 0; t < dc; ++t) {
          const double u = (double)a[t] - (double)b[t];
          dd += u * u;
        }
        if (best < 0 || dd < bd) {
          best = j;
          bd = dd;
        }
      }
      used[(size_t)best] = 1;
      ord[(size_t)i] = best;
      cur = best;
    }
  }
  int rc;
  std::vector<int4> cm[4];
  for (int ci = 0; ci < 4; ++ci) {
    const int mc = 64 >> ci;
    for (int i = 0; i < nl; ++i) {
      const int l = ord[(size_t)i];
      const int64_t n_l = x->h_list_off[l + 1] - x->h_list_off[l];
      for (int64_t m0 = 0; m0 < n_l; m0 += mc)
        cm[ci].push_back(make_int4(l, (int)m0, (int)x->h_list_off[l], (int)n_l));
    }
    x->rr_chunks[ci] = (int)cm[ci].size();
    if ((rc = dmalloc(&x->rr_cmap[ci], std::max<size_t>(cm[ci].size(), 1)))) return rc;
    if (!cm[ci].empty())
      ADN_CUDA(cudaMemcpyAsync(x->rr_cmap[ci], cm[ci].data(), sizeof(int4) * cm[ci].size(),
                               cudaMemcpyHostToDevice, st));
  }
  ADN_CUDA(cudaStreamSynchronize(st));  // the host tables go out of scope
  return ADANNS_OK;
}

}  // namespace adn

using namespace adn;

// Work shape of the FP32 list scan for a batch: queries per thread (tq), the
// query tile (qt) and member ranges per tile (nsplit).
static void fp32_scan_shape(const adanns_index *idx, int64_t B, int d_s, int nprobe, int k, int *tq,
                            int *qt, int *nsplit) {
  const double qpl = (double)B * nprobe / idx->nlist;  // queries per probed list
  int t = tuned_scan_tq(k, d_s, qpl);
  if (t == TUNE_STREAM) t = 0;    // the streaming scan was tuned for this bucket
  if (t == 0 && qpl < 16) t = 1;  // untuned: few queries share a list, small tile
  *tq = t;
  *qt = scan_query_tile(k, t);
  // few work items (a small batch over few lists): split each list into
  // member ranges so every SM has work; each range leaves its own top-k run
  *nsplit = 1;
  const int64_t tiles_est = qpl < *qt ? std::min<int64_t>(idx->nlist, B * nprobe)
                                      : (int64_t)(B * nprobe + *qt - 1) / *qt;
  const int64_t target = (int64_t)num_sms() * 8;
  if (tiles_est > 0 && tiles_est < target)
    *nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((target + tiles_est - 1) / tiles_est,
                                                          (idx->max_list + 255) / 256));
}

extern "C" {

const char *adanns_last_error(void) { return adn::last_error(); }

int adanns_version(void) { return 100; }

int64_t adanns_launch_count(void) { return (int64_t)g_launches.load(); }

int adanns_set_option(int option, int64_t value) { return set_option(option, value); }

int adanns_get_option(int option, int64_t *value) {
  if (!value) return fail(ADANNS_ERR_ARG, "value is NULL");
  if (option < 0 || option >= ADANNS_OPT_COUNT) return fail(ADANNS_ERR_ARG, "unknown option");
  *value = adn::option(option);
  return ADANNS_OK;
}

int adanns_index_create(const float *db, int64_t N, int d, const float *centroids, int nlist,
                        int d_c, const int32_t *assign, int metric, int storage_mask,
                        void *cuda_stream, adanns_index **out) {
  if (!out) return fail(ADANNS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!db || !centroids || !assign) return fail(ADANNS_ERR_ARG, "NULL input");
  if (N < 1 || N > INT32_MAX || d < 1 || nlist < 1 || nlist > 32768)
    return fail(ADANNS_ERR_ARG, "bad sizes");
  int rc;
  if ((rc = check_metric(metric)) || (rc = check_gran(d_c, d, "d_c"))) return rc;
  if (!(storage_mask & ADANNS_STORE_F32)) return fail(ADANNS_ERR_ARG, "storage must include F32");
  if ((rc = check_assignment(assign, N, nlist, S(cuda_stream)))) return rc;
  return make_index(db, N, d, centroids, nlist, d_c, assign, metric, storage_mask, S(cuda_stream),
                    out);
}

int adanns_build_ivf(const float *db, int64_t N, int d, int d_c, int nlist, int niter,
                     int64_t train_n, uint64_t seed, int metric, int storage_mask,
                     double *objective, void *cuda_stream, adanns_index **out) {
  if (!out) return fail(ADANNS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!db) return fail(ADANNS_ERR_ARG, "db is NULL");
  if (N < 1 || N > INT32_MAX || d < 1 || nlist < 1 || nlist > 32768 || niter < 0)
    return fail(ADANNS_ERR_ARG, "bad sizes");
  if (train_n < nlist || train_n > N) return fail(ADANNS_ERR_ARG, "need nlist <= train_n <= N");
  int rc;
  if ((rc = check_metric(metric)) || (rc = check_gran(d_c, d, "d_c"))) return rc;
  if (!(storage_mask & ADANNS_STORE_F32)) return fail(ADANNS_ERR_ARG, "storage must include F32");
  cudaStream_t st = S(cuda_stream);
  const int dcp = pad16(d_c);

  // training sample and Forgy initialisation (seeded, as the oracle defines them)
  std::vector<int64_t> S1 = seeded_sample(seed, N, train_n);
  std::vector<int64_t> S2 = seeded_sample(seed + 1, train_n, nlist);
  Scratch s(st);
  int64_t *d_s1, *d_s2, *cent_off;
  float *tn, *cent, *cent_pm, *kd;
  uint64_t *keys;
  int32_t *asg, *counts, *asg_all;
  double *sums, *obj;
  int *counter, *err;
  if ((rc = s.get(&d_s1, train_n)) || (rc = s.get(&d_s2, nlist)) ||
      (rc = s.get(&tn, (size_t)train_n * dcp)) || (rc = s.get(&cent, (size_t)nlist * d_c)) ||
      (rc = s.get(&cent_pm, (size_t)nlist * dcp)) || (rc = s.get(&keys, train_n)) ||
      (rc = s.get(&asg, train_n)) || (rc = s.get(&counts, nlist)) ||
      (rc = s.get(&sums, (size_t)nlist * d_c)) || (rc = s.get(&obj, 1)) ||
      (rc = s.get(&counter, 1)) || (rc = s.get(&cent_off, 2)) || (rc = s.get(&asg_all, N)) ||
      (rc = s.get(&kd, 1)) || (rc = s.get(&err, 1)))
    return rc;
  ADN_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  ADN_CUDA(cudaMemcpyAsync(d_s1, S1.data(), sizeof(int64_t) * train_n, cudaMemcpyHostToDevice, st));
  ADN_CUDA(cudaMemcpyAsync(d_s2, S2.data(), sizeof(int64_t) * nlist, cudaMemcpyHostToDevice, st));
  const int64_t h_off[2] = {0, (int64_t)nlist};
  ADN_CUDA(cudaMemcpyAsync(cent_off, h_off, sizeof(h_off), cudaMemcpyHostToDevice, st));
  if ((rc = launch_gather_normalize(db, train_n, d, d_s1, d_c, metric, tn, dcp, st))) return rc;
  if ((rc = launch_gather_normalize(tn, nlist, dcp, d_s2, d_c, ADANNS_METRIC_L2, cent, d_c, st)))
    return rc;
  for (int it = 0; it < niter; ++it) {
    if ((rc = centroids_pm(cent, nlist, d_c, cent_pm, st))) return rc;
    if ((rc = nearest_centroid(cent, nlist, d_c, metric, cent_pm, cent_off, tn, train_n, dcp, keys,
                               counter, err, st)))
      return rc;
    if ((rc = launch_sum_keys(keys, train_n, obj, st))) return rc;
    if ((rc = launch_keys_to_result(keys, train_n, 1, nullptr, asg, nullptr, st))) return rc;
    if ((rc = launch_kmeans_update(tn, train_n, dcp, d_c, asg, nlist, sums, counts, cent, st)))
      return rc;
    double J = 0.0;
    ADN_CUDA(cudaMemcpyAsync(&J, obj, sizeof(double), cudaMemcpyDeviceToHost, st));
    ADN_CUDA(cudaStreamSynchronize(st));
    if (objective) objective[it] = J;
  }
  if ((rc = centroids_pm(cent, nlist, d_c, cent_pm, st))) return rc;
  if ((rc = assign_all(db, N, d, d_c, metric, cent, cent_pm, cent_off, nlist, asg_all, nullptr,
                       err, st)))
    return rc;
  {
    int h = 0;
    ADN_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    ADN_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(ADANNS_ERR_TIMEOUT, "a tensor-core pipeline wait timed out in the k-means assignment");
  }
  return make_index(db, N, d, cent, nlist, d_c, asg_all, metric, storage_mask, st, out);
}

int adanns_index_info(const adanns_index *idx, int64_t *N, int *d, int *d_c, int *nlist,
                      int *metric) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (N) *N = idx->N;
  if (d) *d = idx->d;
  if (d_c) *d_c = idx->d_c;
  if (nlist) *nlist = idx->nlist;
  if (metric) *metric = idx->metric;
  return ADANNS_OK;
}

int adanns_index_get_lists(const adanns_index *idx, int64_t *list_off, int32_t *list_ids,
                           void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  cudaStream_t st = S(cuda_stream);
  if (list_off)
    ADN_CUDA(cudaMemcpyAsync(list_off, idx->list_off, sizeof(int64_t) * (idx->nlist + 1),
                             cudaMemcpyDeviceToDevice, st));
  if (list_ids)
    ADN_CUDA(cudaMemcpyAsync(list_ids, idx->list_ids, sizeof(int32_t) * idx->N,
                             cudaMemcpyDeviceToDevice, st));
  return ADANNS_OK;
}

int adanns_index_get_centroids(const adanns_index *idx, float *centroids, void *cuda_stream) {
  if (!idx || !centroids) return fail(ADANNS_ERR_ARG, "NULL argument");
  ADN_CUDA(cudaMemcpyAsync(centroids, idx->centroids, sizeof(float) * idx->nlist * idx->d_c,
                           cudaMemcpyDeviceToDevice, S(cuda_stream)));
  return ADANNS_OK;
}

int adanns_index_status(const adanns_index *idx, void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  cudaStream_t st = S(cuda_stream);
  int h = 0;
  ADN_CUDA(cudaMemcpyAsync(&h, idx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  ADN_CUDA(cudaMemsetAsync(idx->dev_err, 0, sizeof(int), st));
  ADN_CUDA(cudaStreamSynchronize(st));
  if (h & ADANNS_DEVERR_RERANK)
    return fail(ADANNS_ERR_STATE, "rerank found a pair outside its member chunk (skipped)");
  if (h) return fail(ADANNS_ERR_TIMEOUT, "a tensor-core pipeline wait timed out (stage " +
                                             std::to_string(h & 0xff) + ")");
  return ADANNS_OK;
}

}  // extern "C"

namespace adn {
int search_f32_tiled(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                     int nprobe, int k, int64_t *out_ids, float *out_dist, int32_t *out_probes,
                     cudaStream_t st, const QueryBudgets *qb, const int32_t *rows) {
  int rc;
  const int nlist = idx->nlist;
  const int dcp = pad16(d_c), dsp = pad16(d_s);
  int tq, qt, nsplit;
  fp32_scan_shape(idx, B, d_s, nprobe, k, &tq, &qt, &nsplit);
  // slice the batch so that the per-(query, probe) partial results stay ~2 GiB
  const int64_t per_q =
      (int64_t)nprobe * nsplit * k * 8 + (int64_t)(dcp + dsp) * 4 + nprobe * 24;
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, (2ll << 30) / per_q));
  const int64_t max_tiles = (Bc * nprobe + qt - 1) / qt + nlist;
  Scratch s(st);
  float *qc, *qs;
  uint64_t *ckeys, *pkeys;
  int32_t *lcnt, *lbeg, *lfill, *tbeg, *pair_q, *pair_out, *tl, *tb, *tc;
  int *ntiles, *counter;
  if ((rc = s.get(&qc, (size_t)Bc * dcp)) || (rc = s.get(&qs, (size_t)Bc * dsp)) ||
      (rc = s.get(&ckeys, (size_t)Bc * nprobe)) || (rc = s.get(&pkeys, (size_t)Bc * nprobe * nsplit * k)) ||
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
    const QueryBudgets bq = qb ? qb->at(b0) : QueryBudgets{};
    const int32_t *rws = rows ? rows + b0 : nullptr;
    {
      StageTimer t(ST_PREP, st);
      if ((rc = launch_prep_queries(rws ? queries : queries + b0 * idx->d, nb, idx->d, d_c, d_s,
                                    idx->metric, qc, dcp, qs, dsp, st, nullptr, rws)))
        return rc;
    }
    // cluster mapping: nprobe nearest centroids at d_c
    ADN_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st));
    {
      StageTimer t(ST_COARSE, st);
      if ((rc = run_coarse(idx, qc, dcp, nb, d_c, nprobe, ckeys, counter, st))) return rc;
      if ((rc = launch_mask_probes(ckeys, nb, nprobe, bq.np, st))) return rc;
    }
    {
      StageTimer t(ST_INVERT, st);
      if ((rc = launch_invert_probes(ckeys, nb, nprobe, nlist, qt, lcnt, lbeg, lfill, tbeg, pair_q,
                                     pair_out, tl, tb, tc, ntiles,
                                     out_probes ? out_probes + b0 * nprobe : nullptr, st)))
        return rc;
    }
    // linear scan of the probed lists at d_s
    ScanArgs l{};
    l.xpm = idx->xpm;
    l.d_pad = idx->d_pad;
    l.dims = d_s;
    l.list_off = idx->list_off;
    l.list_ids = idx->list_ids;
    l.mscale = mscale;
    l.qn = qs;
    l.ldq = dsp;
    l.tile_list = tl;
    l.tile_beg = tb;
    l.tile_cnt = tc;
    l.ntiles_dev = ntiles;
    l.counter = counter + 1;
    l.pair_q = pair_q;
    l.pair_out = pair_out;
    l.k = k;
    l.out_keys = pkeys;
    l.tq = tq;
    l.nsplit = nsplit;
    {
      StageTimer t(ST_SCAN, st);
      if ((rc = launch_scan_f32(l, st))) return rc;
    }
    {
      StageTimer t(ST_MERGE, st);
      MergeMask mm;
      if (bq.np) {
        mm.ckeys = ckeys;
        mm.nsplit = nsplit;
      }
      mm.kq = bq.k;
      mm.orow = rws;
      if ((rc = launch_merge(pkeys, nb, nprobe * nsplit, k, rws ? out_ids : out_ids + b0 * k,
                             rws ? out_dist : out_dist + b0 * k, st, mm)))
        return rc;
    }
  }
  return ADANNS_OK;
}

int64_t stream_scratch_bytes(const adanns_index *idx, int64_t B, int d_c, int d_s, int nprobe,
                             int k) {
  const int64_t per_q = max_probe_members(idx, nprobe) * 4 + (int64_t)(pad16(d_c) + pad16(d_s)) * 4 +
                        (int64_t)k * 8 + (int64_t)nprobe * 40 + 16;
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, scratch_budget() / per_q));
  return Bc * per_q + (int64_t)idx->nlist * 64 + (16ll << 20);
}
}  // namespace adn

extern "C" {
int64_t adanns_search_scratch_bytes(const adanns_index *idx, int64_t B, int d_c, int d_s,
                                    int nprobe, int k, int storage, int rerank_k) {
  if (!idx || B < 0 || nprobe < 1 || k < 1) return -1;
  const int dcp = pad16(d_c), dsp = pad16(d_s);
  if (storage == ADANNS_STORE_BF16 || storage == ADANNS_STORE_FP8E4M3) {
    const int epb = storage == ADANNS_STORE_FP8E4M3 ? 128 : 64;
    const int64_t nkb = (d_s + epb - 1) / epb;
    const int64_t kk = rerank_k > k ? rerank_k : k;
    const int64_t seg_q = (int64_t)nprobe * (((int64_t)idx->max_list + 7) & ~7ll);
    const int64_t per_q = seg_q * 2 + (int64_t)nprobe * (nkb * 128 * 128 / 128 + 32) +
                          (int64_t)(dcp + dsp) * 4 + nkb * 128 + kk * 8 + 64 + kk * 40;
    const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, scratch_budget() / per_q));
    return Bc * per_q + (int64_t)idx->nlist * 64 + (64ll << 20);
  }
  if (fp32_stream_enabled((double)B * nprobe / idx->nlist, nprobe, k, d_s))
    return stream_scratch_bytes(idx, B, d_c, d_s, nprobe, k);
  int tq, qt, nsplit;
  fp32_scan_shape(idx, B, d_s, nprobe, k, &tq, &qt, &nsplit);
  const int64_t per_q =
      (int64_t)nprobe * nsplit * k * 8 + (int64_t)(dcp + dsp) * 4 + nprobe * 24;
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, (2ll << 30) / per_q));
  return Bc * per_q + (int64_t)idx->nlist * 64 + (16ll << 20);
}

void adanns_index_free(adanns_index *idx) {
  if (!idx) return;
  cudaDeviceSynchronize();
  free_index(idx);
}

int adanns_kmeans_assign(const float *points, int64_t n, int ld, int dim, int metric,
                         const float *centroids, int nc, int32_t *out_assign, float *out_dist,
                         void *cuda_stream) {
  if (!points || !centroids || !out_assign) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (n < 0 || n > INT32_MAX || nc < 1 || ld < dim) return fail(ADANNS_ERR_ARG, "bad sizes");
  int rc;
  if ((rc = check_metric(metric)) || (rc = check_gran(dim, ld, "dim"))) return rc;
  if (n == 0) return ADANNS_OK;
  cudaStream_t st = S(cuda_stream);
  Scratch s(st);
  float *cpm;
  int64_t *coff;
  if ((rc = s.get(&cpm, (size_t)nc * pad16(dim))) || (rc = s.get(&coff, 2))) return rc;
  const int64_t h_off[2] = {0, (int64_t)nc};
  ADN_CUDA(cudaMemcpyAsync(coff, h_off, sizeof(h_off), cudaMemcpyHostToDevice, st));
  if ((rc = centroids_pm(centroids, nc, dim, cpm, st))) return rc;
  int *err;
  if ((rc = s.get(&err, 1))) return rc;
  ADN_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  if ((rc = assign_all(points, n, ld, dim, metric, centroids, cpm, coff, nc, out_assign, out_dist,
                       err, st)))
    return rc;
  int h = 0;
  ADN_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  ADN_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(ADANNS_ERR_TIMEOUT, "a tensor-core pipeline wait timed out in the assignment");
  return ADANNS_OK;
}

int adanns_kmeans_update(const float *points, int64_t n, int ld, int dim, int metric,
                         const int32_t *assign, int nc, float *centroids, void *cuda_stream) {
  if (!points || !assign || !centroids) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (n < 0 || n > INT32_MAX || nc < 1 || ld < dim) return fail(ADANNS_ERR_ARG, "bad sizes");
  int rc;
  if ((rc = check_metric(metric)) || (rc = check_gran(dim, ld, "dim"))) return rc;
  cudaStream_t st = S(cuda_stream);
  Scratch s(st);
  float *pn;
  double *sums;
  int32_t *counts;
  if ((rc = s.get(&pn, (size_t)std::max<int64_t>(n, 1) * dim)) ||
      (rc = s.get(&sums, (size_t)nc * dim)) || (rc = s.get(&counts, nc)))
    return rc;
  if ((rc = launch_gather_normalize(points, n, ld, nullptr, dim, metric, pn, dim, st))) return rc;
  return launch_kmeans_update(pn, n, dim, dim, assign, nc, sums, counts, centroids, st);
}

int adanns_search_ivf(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                      int d_s, int nprobe, int k, int storage, int rerank_k, int64_t *out_ids,
                      float *out_dist, int32_t *out_probes, void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (B < 0 || B > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad batch size");
  if (B > 0 && (!queries || !out_ids || !out_dist)) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (gran_index(d_c) < 0 || d_c > idx->d_c)
    return fail(ADANNS_ERR_DIM, "d_c must be an MR granularity <= the index's clustering prefix " +
                                    std::to_string(idx->d_c));
  int rc;
  if ((rc = check_gran(d_s, idx->d, "d_s"))) return rc;
  if (nprobe < 1 || nprobe > idx->nlist) return fail(ADANNS_ERR_ARG, "need 1 <= nprobe <= nlist");
  if (k < 1 || k > 1024) return fail(ADANNS_ERR_ARG, "need 1 <= k <= 1024");
  if (storage == ADANNS_STORE_BF16 || storage == ADANNS_STORE_FP8E4M3) {
    const int which = storage == ADANNS_STORE_BF16 ? 0 : 1;
    if (!idx->lowp[which]) return fail(ADANNS_ERR_STATE, "the index has no such storage tier");
    if (idx->metric != ADANNS_METRIC_L2_PREFIXNORM)
      return fail(ADANNS_ERR_STATE, "low-precision search needs the prefix-normalised metric");
    if (rerank_k < k || rerank_k > 2048)
      return fail(ADANNS_ERR_ARG, "low-precision search needs k <= rerank_k <= 2048");
    if (nprobe > 128) return fail(ADANNS_ERR_ARG, "low-precision search needs nprobe <= 128");
    if (B == 0) return ADANNS_OK;
    return search_mixed(idx, queries, B, d_c, d_s, nprobe, k, which, rerank_k, out_ids, out_dist,
                        out_probes, S(cuda_stream));
  }
  if (storage != ADANNS_STORE_F32) return fail(ADANNS_ERR_ARG, "unknown storage tier");
  if (rerank_k != 0) return fail(ADANNS_ERR_ARG, "rerank_k must be 0 for the FP32 scan");
  if (B == 0) return ADANNS_OK;
  cudaStream_t st = S(cuda_stream);
  if (fp32_stream_enabled((double)B * nprobe / idx->nlist, nprobe, k, d_s))
    return search_f32_stream(idx, queries, B, d_c, d_s, nprobe, k, out_ids, out_dist, out_probes,
                             st);
  return search_f32_tiled(idx, queries, B, d_c, d_s, nprobe, k, out_ids, out_dist, out_probes,
                          st);
}

int adanns_search_ivf_budgets(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                              const int32_t *d_s, const int32_t *nprobe, const int32_t *k,
                              int k_max, int storage, int rerank_k, int64_t *out_ids,
                              float *out_dist, void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (B < 0 || B > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad batch size");
  if (B > 0 && (!queries || !out_ids || !out_dist || !d_s || !nprobe || !k))
    return fail(ADANNS_ERR_ARG, "NULL argument");
  if (gran_index(d_c) < 0 || d_c > idx->d_c)
    return fail(ADANNS_ERR_DIM, "d_c must be an MR granularity <= the index's clustering prefix " +
                                    std::to_string(idx->d_c));
  if (k_max < 1 || k_max > 1024) return fail(ADANNS_ERR_ARG, "need 1 <= k_max <= 1024");
  const bool lowp = storage == ADANNS_STORE_BF16 || storage == ADANNS_STORE_FP8E4M3;
  if (!lowp && storage != ADANNS_STORE_F32) return fail(ADANNS_ERR_ARG, "unknown storage tier");
  const int np_cap = lowp ? 128 : 256;
  int ds_max = 0, np_max = 0, rc;
  int64_t np_sum = 0;
  // one staging array: d_s, granularity index, nprobe, k of every query, then
  // the queries in d_s order with their nprobe and k (the tiled FP32 groups)
  std::vector<int32_t> h((size_t)B * 7);
  for (int64_t i = 0; i < B; ++i) {
    const std::string at = " (query " + std::to_string(i) + ")";
    if ((rc = check_gran(d_s[i], idx->d, "d_s"))) return fail(rc, adanns_last_error() + at);
    if (nprobe[i] < 1 || nprobe[i] > idx->nlist || nprobe[i] > np_cap)
      return fail(ADANNS_ERR_ARG, "need 1 <= nprobe <= min(nlist, " + std::to_string(np_cap) +
                                      ")" + at);
    if (k[i] < 1 || k[i] > k_max) return fail(ADANNS_ERR_ARG, "need 1 <= k <= k_max" + at);
    if (lowp && d_s[i] != d_s[0])
      return fail(ADANNS_ERR_ARG, "the low-precision tiers need one d_s per batch" + at);
    ds_max = std::max(ds_max, (int)d_s[i]);
    np_max = std::max(np_max, (int)nprobe[i]);
    np_sum += nprobe[i];
    h[(size_t)i] = d_s[i];
    h[(size_t)(B + i)] = gran_index(d_s[i]);
    h[(size_t)(2 * B + i)] = nprobe[i];
    h[(size_t)(3 * B + i)] = k[i];
  }
  int which = 0;
  if (lowp) {
    which = storage == ADANNS_STORE_BF16 ? 0 : 1;
    if (!idx->lowp[which]) return fail(ADANNS_ERR_STATE, "the index has no such storage tier");
    if (idx->metric != ADANNS_METRIC_L2_PREFIXNORM)
      return fail(ADANNS_ERR_STATE, "low-precision search needs the prefix-normalised metric");
    if (rerank_k < k_max || rerank_k > 2048)
      return fail(ADANNS_ERR_ARG, "low-precision search needs k_max <= rerank_k <= 2048");
  } else if (rerank_k != 0) {
    return fail(ADANNS_ERR_ARG, "rerank_k must be 0 for the FP32 scan");
  }
  if (B == 0) return ADANNS_OK;
  // FP32 with many queries per probed list: the tiled scan, one launch
  // sequence per distinct d_s over that group of queries (rows in place)
  const bool tiled = !lowp && !fp32_stream_enabled((double)np_sum / idx->nlist, np_max);
  std::vector<std::pair<int64_t, int64_t>> grp;  // [begin, end) of each d_s group in the order
  if (tiled) {
    std::vector<int32_t> perm((size_t)B);
    for (int64_t i = 0; i < B; ++i) perm[(size_t)i] = (int32_t)i;
    std::stable_sort(perm.begin(), perm.end(),
                     [&](int32_t a, int32_t b) { return d_s[a] < d_s[b]; });
    for (int64_t i = 0; i < B; ++i) {
      const int32_t r = perm[(size_t)i];
      h[(size_t)(4 * B + i)] = r;
      h[(size_t)(5 * B + i)] = nprobe[r];
      h[(size_t)(6 * B + i)] = k[r];
      if (i == 0 || d_s[r] != d_s[perm[(size_t)i - 1]]) grp.push_back({i, i + 1});
      else grp.back().second = i + 1;
    }
  }
  cudaStream_t st = S(cuda_stream);
  Scratch s(st);
  int32_t *dq;
  if ((rc = s.get(&dq, h.size()))) return rc;
  // pageable source: staged by the copy call itself, so h may go when it returns
  ADN_CUDA(cudaMemcpyAsync(dq, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  QueryBudgets qb;
  qb.ds = dq;
  qb.gi = dq + B;
  qb.np = dq + 2 * B;
  qb.k = dq + 3 * B;
  if (lowp) {
    qb.ds = qb.gi = nullptr;  // one d_s for the batch
    return search_mixed(idx, queries, B, d_c, ds_max, np_max, k_max, which, rerank_k, out_ids,
                        out_dist, nullptr, st, &qb);
  }
  if (tiled) {
    for (const auto &g : grp) {
      const int32_t *perm = dq + 4 * B + g.first;
      int gnp = 0;
      for (int64_t i = g.first; i < g.second; ++i)
        gnp = std::max(gnp, (int)h[(size_t)(5 * B + i)]);
      QueryBudgets gb;
      gb.np = dq + 5 * B + g.first;
      gb.k = dq + 6 * B + g.first;
      if ((rc = search_f32_tiled(idx, queries, g.second - g.first, d_c,
                                 d_s[h[(size_t)(4 * B + g.first)]], gnp, k_max, out_ids, out_dist,
                                 nullptr, st, &gb, perm)))
        return rc;
    }
    return ADANNS_OK;
  }
  return search_f32_stream(idx, queries, B, d_c, ds_max, np_max, k_max, out_ids, out_dist, nullptr,
                           st, &qb);
}

}  // extern "C"
