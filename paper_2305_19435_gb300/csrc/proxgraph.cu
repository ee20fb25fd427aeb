// Low-dimensional graph shortlist with a high-dimensional rerank: the
// AdANNS-DiskANN composite of Sec. 4.3 ("AdANNS for Composite Indices") --
// the search graph is formed with a low-d MR and its shortlist is re-ranked
// with a high-d MR.
//
// Build (one pass, DiskANN-style pruned proximity graph at the d_g prefix):
//   1. every row's K nearest other rows: a brute-force sweep of the FP32 list
//      scan over one list holding all rows (fused top-(K+1), the row itself
//      dropped);
//   2. robust prune of each candidate list with factor alpha to at most R
//      out-neighbours (one warp per row);
//   3. every edge p -> c offers p to c (counting sort by target); a row whose
//      own and offered neighbours exceed R is pruned again over their union
//      sorted by (distance, id) (one CTA per row);
//   4. entry point: the row nearest to the FP64 mean of the rows.
// Search (one warp per query): best-first with a bounded candidate list of L
// entries in shared memory -- expand the nearest entry not yet expanded, score
// its neighbours that are not in the list (one lane each), keep the L nearest
// by (distance, id) -- until every entry is expanded; then the rerank_k
// nearest are re-scored with the exact FP32 distance at d_s and the k best
// returned.  All distances are FP32 in difference form.
#include <algorithm>
#include <vector>

#include "devutil.cuh"
#include "internal.cuh"

struct adanns_graph {
  int64_t N = 0;
  int d = 0, d_g = 0, dg_pad = 0, R = 0, metric = 0;
  int64_t entry = 0;
  float *xg = nullptr;     // N x dg_pad: P_dg of every row (id order)
  int32_t *nbr = nullptr;  // N x R neighbours, -1 padding, each row by (distance, id)
  float *rows = nullptr;   // N x d FP32 rows (id order), for the rerank
  int *dev_err = nullptr;
};

namespace adn {
namespace {

constexpr int GR_MAXR = 64;      // out-degree limit
constexpr int GR_MAXK = 256;     // candidate list limit of the build
constexpr int GR_MAXDG = 64;     // graph dimension limit (one lane scores a whole row)
constexpr int GR_MAXL = 512;     // search list limit
constexpr int GR_UCAP = 4096;    // own + offered neighbours of one row in the final prune
constexpr int ERR_HUB = 0x200;   // status bit: a row was offered more than GR_UCAP edges

__device__ __forceinline__ float sqdist(const float *a, const float *b, int m) {
  float acc = 0.f;
  for (int j = 0; j < m; ++j) {
    const float t = a[j] - b[j];
    acc = fmaf(t, t, acc);
  }
  return acc;
}

__device__ __forceinline__ uint64_t gkey(float d, int32_t id) {
  return ((uint64_t)__float_as_uint(d) << 32) | (uint32_t)id;
}

// ---------------------------------------------------------------- build
// knn[p][0:K] from the sweep's sorted (K + 1) keys: the row itself (or, among
// rows at distance 0, the last one) is left out
__global__ void knn_drop_self_kernel(const uint64_t *__restrict__ keys, int64_t N, int K,
                                     int32_t *__restrict__ knn, float *__restrict__ kd) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const uint64_t *k = keys + p * (K + 1);
  int w = 0;
  bool dropped = false;
  for (int r = 0; r <= K && w < K; ++r) {
    const uint64_t v = k[r];
    const int32_t id = v == KEY_MAX ? -1 : (int32_t)(uint32_t)(v & 0xffffffffu);
    if (!dropped && id == (int32_t)p) {
      dropped = true;
      continue;
    }
    knn[p * K + w] = id;
    kd[p * K + w] = id < 0 ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(v >> 32));
    ++w;
  }
  for (; w < K; ++w) {
    knn[p * K + w] = -1;
    kd[p * K + w] = __int_as_float(0x7f800000);
  }
}

// one warp per row: robust prune of its K candidates (sorted by (distance, id))
__global__ void prune_kernel(const float *__restrict__ xg, int ldg, int d_g,
                             const int32_t *__restrict__ knn, const float *__restrict__ kd, int K,
                             int64_t N, float alpha, int R, int32_t *__restrict__ fwd,
                             int32_t *__restrict__ nfwd) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (p >= N) return;
  constexpr int PER = GR_MAXK / 32;
  int32_t id[PER];
  float dp[PER];
  bool alive[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int r = u * 32 + lane;
    id[u] = r < K ? knn[p * K + r] : -1;
    dp[u] = r < K ? kd[p * K + r] : 0.f;
    alive[u] = id[u] >= 0 && id[u] != (int32_t)p;
  }
  int nout = 0;
  for (int r0 = 0; r0 < K && nout < R; ++r0) {
    // candidate r0 is the nearest alive one when it is alive (list order)
    const int u0 = r0 >> 5;
    bool al = false;
    int32_t c = -1;
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (u == u0) {
        al = alive[u];
        c = id[u];
      }
    al = __shfl_sync(0xffffffffu, al, r0 & 31);
    c = __shfl_sync(0xffffffffu, c, r0 & 31);
    if (!al) continue;
    if (lane == 0) fwd[p * R + nout] = c;
    ++nout;
    const float *xc = xg + (int64_t)c * ldg;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int r = u * 32 + lane;
      if (r == r0) alive[u] = false;
      if (r > r0 && alive[u]) {
        const float dcv = alpha * sqdist(xc, xg + (int64_t)id[u] * ldg, d_g);
        if (dcv <= dp[u]) alive[u] = false;
      }
    }
  }
  for (int r = nout + lane; r < R; r += 32) fwd[p * R + r] = -1;
  if (lane == 0) nfwd[p] = nout;
}

__global__ void offer_count_kernel(const int32_t *__restrict__ fwd, int64_t n, int32_t *cnt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t c = fwd[e];
  if (c >= 0) atomicAdd(&cnt[c], 1);
}

__global__ void offer_fill_kernel(const int32_t *__restrict__ fwd, int64_t n, int R,
                                  int32_t *__restrict__ cursor, int32_t *__restrict__ rev) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t c = fwd[e];
  if (c >= 0) rev[atomicAdd(&cursor[c], 1)] = (int32_t)(e / R);
}

// one CTA per row q: union of own and offered neighbours by (distance, id),
// duplicates dropped; kept whole when it fits R, else robust-pruned to R
constexpr int FIN_THREADS = 256;
__global__ void __launch_bounds__(FIN_THREADS) final_prune_kernel(
    const float *__restrict__ xg, int ldg, int d_g, const int32_t *__restrict__ fwd,
    const int32_t *__restrict__ nfwd, const int32_t *__restrict__ roff,
    const int32_t *__restrict__ rev, int64_t N, float alpha, int R, int32_t *__restrict__ out,
    int *__restrict__ err) {
  __shared__ uint64_t u[GR_UCAP];
  __shared__ int s_n;
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x;
  const int nf = nfwd[q];
  const int r0 = roff[q], nr = roff[q + 1] - r0;
  int nu = nf + nr;
  if (nu > GR_UCAP) {  // a hub beyond the buffer: report, keep its own list
    if (tid == 0) atomicOr(err, ERR_HUB);
    for (int r = tid; r < R; r += FIN_THREADS) out[q * R + r] = fwd[q * R + r];
    return;
  }
  const float *xq = xg + q * ldg;
  for (int i = tid; i < nu; i += FIN_THREADS) {
    const int32_t c = i < nf ? fwd[q * R + i] : rev[r0 + i - nf];
    u[i] = gkey(sqdist(xq, xg + (int64_t)c * ldg, d_g), c);
  }
  int P = 1;
  while (P < nu) P <<= 1;
  for (int i = nu + tid; i < P; i += FIN_THREADS) u[i] = KEY_MAX;
  __syncthreads();
  // bitonic sort of P keys
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < P; i += FIN_THREADS) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const uint64_t a = u[i], b = u[j];
          if ((a > b) == up) {
            u[i] = b;
            u[j] = a;
          }
        }
      }
      __syncthreads();
    }
  // drop duplicates (equal keys are adjacent)
  if (tid == 0) {
    int w = 0;
    for (int i = 0; i < nu; ++i)
      if (w == 0 || u[i] != u[w - 1]) u[w++] = u[i];
    s_n = w;
  }
  __syncthreads();
  nu = s_n;
  if (nu <= R) {
    for (int r = tid; r < R; r += FIN_THREADS)
      out[q * R + r] = r < nu ? (int32_t)(uint32_t)(u[r] & 0xffffffffu) : -1;
    return;
  }
  // robust prune over the sorted union: a pruned entry is overwritten with
  // the empty key
  int nout = 0;
  for (int i = 0; i < nu && nout < R; ++i) {
    __syncthreads();
    if (u[i] == KEY_MAX) continue;  // uniform: every thread reads the same slot
    const int32_t c = (int32_t)(uint32_t)(u[i] & 0xffffffffu);
    if (tid == 0) out[q * R + nout] = c;
    ++nout;
    const float *xc = xg + (int64_t)c * ldg;
    __syncthreads();
    for (int j = i + 1 + tid; j < nu; j += FIN_THREADS) {
      const uint64_t v = u[j];
      if (v == KEY_MAX) continue;
      const int32_t vid = (int32_t)(uint32_t)(v & 0xffffffffu);
      const float dpv = __uint_as_float((uint32_t)(v >> 32));
      if (alpha * sqdist(xc, xg + (int64_t)vid * ldg, d_g) <= dpv) u[j] = KEY_MAX;
    }
  }
  __syncthreads();
  for (int r = nout + tid; r < R; r += FIN_THREADS) out[q * R + r] = -1;
}

// FP64 coordinate sums of the rows (one thread per (block of rows, coordinate))
__global__ void row_sum_kernel(const float *__restrict__ xg, int ldg, int d_g, int64_t N,
                               double *__restrict__ sum) {
  const int j = threadIdx.x;
  if (j >= d_g) return;
  double acc = 0.0;
  for (int64_t p = blockIdx.x; p < N; p += gridDim.x) acc += (double)xg[p * ldg + j];
  atomicAdd(&sum[j], acc);
}

__global__ void entry_kernel(const float *__restrict__ xg, int ldg, int d_g, int64_t N,
                             const double *__restrict__ sum, unsigned long long *__restrict__ best) {
  __shared__ float mean[GR_MAXDG];
  if (threadIdx.x < d_g) mean[threadIdx.x] = (float)(sum[threadIdx.x] / (double)N);
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  atomicMin(best, (unsigned long long)gkey(sqdist(xg + p * ldg, mean, d_g), (int32_t)p));
}

// ---------------------------------------------------------------- search
constexpr int GS_WARPS = 4;

struct GsArgs {
  const float *xg;
  int ldg, d_g;
  const int32_t *nbr;
  int R;
  int64_t entry, N;
  const float *qg;
  int ldq;
  int64_t B;
  int L, kk;
  int64_t *short_ids;  // [B][kk], -1 padding
  int64_t *nexp;       // optional [B]
};

// one warp per query; the list (keys sorted ascending, expanded flags) and a
// merge buffer live in shared memory
__global__ void __launch_bounds__(GS_WARPS * 32) graph_search_kernel(GsArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t qi = (int64_t)blockIdx.x * GS_WARPS + warp;
  const int L = a.L, cap = L + GR_MAXR;
  uint64_t *lst = (uint64_t *)smem + (size_t)warp * 2 * cap;  // [cap] list, [cap] merge
  uint64_t *mrg = lst + cap;
  unsigned char *done = smem + (size_t)GS_WARPS * 2 * cap * 8 + (size_t)warp * cap;
  float *qv = (float *)(smem + (size_t)GS_WARPS * 2 * cap * 8 + (size_t)GS_WARPS * cap) +
              (size_t)warp * GR_MAXDG;
  if (qi >= a.B) return;
  for (int j = lane; j < a.d_g; j += 32) qv[j] = a.qg[qi * a.ldq + j];
  __syncwarp();
  int n = 1;
  if (lane == 0) {
    lst[0] = gkey(sqdist(qv, a.xg + a.entry * a.ldg, a.d_g), (int32_t)a.entry);
    done[0] = 0;
  }
  __syncwarp();
  int64_t nexp = 0;
  for (int64_t it = 0; it < a.N; ++it) {
    // the nearest entry not yet expanded (the list is sorted)
    int sel = -1;
    for (int b = 0; b < n; b += 32) {
      const unsigned m = __ballot_sync(0xffffffffu, b + lane < n && !done[b + lane]);
      if (m) {
        sel = b + __ffs(m) - 1;
        break;
      }
    }
    if (sel < 0) break;
    const int32_t v = (int32_t)(uint32_t)(lst[sel] & 0xffffffffu);
    __syncwarp();
    if (lane == 0) done[sel] = 1;
    ++nexp;
    // neighbours not in the list, scored by one lane each.  A neighbour's key
    // (distance bits, id) is the same every time it is scored and keys are
    // unique, so it is in the (sorted) list exactly when its key is: a binary
    // search instead of a scan of the list
    int nn = 0;
    for (int r0 = 0; r0 < a.R; r0 += 32) {
      const int r = r0 + lane;
      const int32_t u = r < a.R ? a.nbr[(int64_t)v * a.R + r] : -1;
      bool in = u < 0;
      uint64_t key = KEY_MAX;
      if (!in) {
        key = gkey(sqdist(qv, a.xg + (int64_t)u * a.ldg, a.d_g), u);
        int lo = 0, hi = n;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (lst[mid] < key) lo = mid + 1; else hi = mid;
        }
        in = lo < n && lst[lo] == key;
      }
      const unsigned m = __ballot_sync(0xffffffffu, !in);
      if (!in) mrg[nn + __popc(m & lanemask_lt())] = key;
      nn += __popc(m);
    }
    __syncwarp();
    if (nn == 0) continue;
    // new keys sorted, then merged with the list; the L smallest stay
    warp_sort(mrg, nn);
    __syncwarp();
    // merge path: each output slot o < min(n + nn, L) takes its element
    const int tot = min(n + nn, L);
    uint64_t ok[(GR_MAXL + GR_MAXR) / 32];
    unsigned char of[(GR_MAXL + GR_MAXR) / 32];
#pragma unroll
    for (int s = 0; s < (GR_MAXL + GR_MAXR) / 32; ++s) {
      const int o = s * 32 + lane;
      ok[s] = KEY_MAX;
      of[s] = 0;
      if (o < tot) {
        // the number of list keys among the first o + 1 outputs: the largest i
        // with i + j = o + 1, lst[i - 1] < mrg[j] (binary search on i)
        int lo = max(0, o + 1 - nn), hi = min(o + 1, n);
        while (lo < hi) {
          const int i = (lo + hi + 1) >> 1;
          const int j = o + 1 - i;
          if (j >= nn || lst[i - 1] < mrg[j]) lo = i; else hi = i - 1;
        }
        const int i = lo, j = o + 1 - i;  // o-th output = the larger of lst[i-1], mrg[j-1]
        const bool from_l = j == 0 || (i > 0 && lst[i - 1] > mrg[j - 1]);
        ok[s] = from_l ? lst[i - 1] : mrg[j - 1];
        of[s] = from_l ? done[i - 1] : 0;
      }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < (GR_MAXL + GR_MAXR) / 32; ++s) {
      const int o = s * 32 + lane;
      if (o < tot) {
        lst[o] = ok[s];
        done[o] = of[s];
      }
    }
    __syncwarp();
    n = tot;
  }
  for (int r = lane; r < a.kk; r += 32)
    a.short_ids[qi * a.kk + r] = r < n ? (int64_t)(uint32_t)(lst[r] & 0xffffffffu) : -1;
  if (a.nexp && lane == 0) a.nexp[qi] = nexp;
}

// per query (one warp): exact FP32 distance at d_s of each shortlisted row
// (difference form against the row's own normalised prefix), the k best
__global__ void graph_rerank_kernel(const int64_t *__restrict__ cand, int kk, int64_t B,
                                    const float *__restrict__ qs, int ldq, int d_s,
                                    const float *__restrict__ rows, int d, int metric, int k,
                                    int64_t *__restrict__ out_ids, float *__restrict__ out_dist) {
  extern __shared__ uint64_t rk[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * 4 + warp;
  if (q >= B) return;
  uint64_t *buf = rk + (size_t)warp * kk;
  const float *qr = qs + q * ldq;
  int n = 0;
  for (int r = 0; r < kk; ++r) {
    const int64_t id = cand[q * kk + r];
    if (id < 0) break;
    const float *x = rows + id * (int64_t)d;
    float s2 = 0.f;
    for (int j = lane; j < d_s; j += 32) s2 = fmaf(x[j], x[j], s2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const float nu = metric == ADANNS_METRIC_L2_PREFIXNORM ? (s2 > 0.f ? 1.f / sqrtf(s2) : 0.f) : 1.f;
    float acc = 0.f;
    for (int j = lane; j < d_s; j += 32) {
      const float t = fmaf(-nu, x[j], qr[j]);
      acc = fmaf(t, t, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) buf[n] = gkey(acc, (int32_t)id);
    ++n;
  }
  __syncwarp();
  warp_sort(buf, n);
  for (int r = lane; r < k; r += 32) {
    const bool ok = r < n;
    out_ids[q * k + r] = ok ? (int64_t)(uint32_t)(buf[r] & 0xffffffffu) : -1;
    out_dist[q * k + r] = ok ? __uint_as_float((uint32_t)(buf[r] >> 32)) : __int_as_float(0x7f800000);
  }
}

// flag (bit 1) any neighbour id outside [-1, N)
__global__ void graph_check_kernel(const int32_t *__restrict__ nbr, int64_t n, int64_t N,
                                   int *__restrict__ bad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n && (nbr[e] < -1 || (int64_t)nbr[e] >= N)) atomicOr(bad, 1);
}

template <class T>
int gmalloc(T **p, size_t count) {
  if (cudaMalloc((void **)p, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ADANNS_ERR_OOM, "graph allocation failed");
  }
  return ADANNS_OK;
}

void free_graph(adanns_graph *g) {
  if (!g) return;
  cudaFree(g->xg);
  cudaFree(g->nbr);
  cudaFree(g->rows);
  cudaFree(g->dev_err);
  delete g;
}

int check_graph_shape(int64_t N, int d, int d_g, int R, int metric) {
  if (N < 2 || N > INT32_MAX || d < 1) return fail(ADANNS_ERR_ARG, "bad sizes");
  if (gran_index(d_g) < 0 || d_g > d || d_g > GR_MAXDG)
    return fail(ADANNS_ERR_DIM, "d_g must be an MR granularity <= min(d, 64)");
  if (R < 1 || R > GR_MAXR) return fail(ADANNS_ERR_ARG, "need 1 <= R <= 64");
  if (metric != ADANNS_METRIC_L2 && metric != ADANNS_METRIC_L2_PREFIXNORM)
    return fail(ADANNS_ERR_ARG, "unknown metric");
  return ADANNS_OK;
}

// a graph shell holding the rows and their d_g prefixes
int make_shell(const float *db, int64_t N, int d, int d_g, int R, int metric, cudaStream_t st,
               adanns_graph **out) {
  adanns_graph *g = new adanns_graph();
  g->N = N;
  g->d = d;
  g->d_g = d_g;
  g->dg_pad = pad16(d_g);
  g->R = R;
  g->metric = metric;
  int rc;
  if ((rc = gmalloc(&g->xg, (size_t)N * g->dg_pad)) || (rc = gmalloc(&g->nbr, (size_t)N * R)) ||
      (rc = gmalloc(&g->rows, (size_t)N * d)) || (rc = gmalloc(&g->dev_err, 1))) {
    free_graph(g);
    return rc;
  }
  if (cudaMemcpyAsync(g->rows, db, sizeof(float) * N * d, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(g->dev_err, 0, sizeof(int), st) != cudaSuccess) {
    free_graph(g);
    return cuda_fail(cudaGetLastError(), "graph copy");
  }
  if ((rc = launch_gather_normalize(db, N, d, nullptr, d_g, metric, g->xg, g->dg_pad, st))) {
    free_graph(g);
    return rc;
  }
  *out = g;
  return ADANNS_OK;
}

}  // namespace
}  // namespace adn

using namespace adn;

extern "C" {

int adanns_graph_build(const float *db, int64_t N, int d, int d_g, int K, int R, float alpha,
                       int metric, void *cuda_stream, adanns_graph **out) {
  if (!out) return fail(ADANNS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!db) return fail(ADANNS_ERR_ARG, "db is NULL");
  int rc;
  if ((rc = check_graph_shape(N, d, d_g, R, metric))) return rc;
  if (K < 1 || K > GR_MAXK || K >= N) return fail(ADANNS_ERR_ARG, "need 1 <= K <= 256, K < N");
  if (!(alpha >= 1.f) || !(alpha < 3.0e38f)) return fail(ADANNS_ERR_ARG, "need alpha >= 1");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  adanns_graph *g = nullptr;
  if ((rc = make_shell(db, N, d, d_g, R, metric, st, &g))) return rc;
  auto bail = [&](int code) {
    cudaStreamSynchronize(st);
    free_graph(g);
    return code;
  };
  {
    Scratch s(st);
    float *xpm, *kd;
    int64_t *off;
    uint64_t *keys;
    int32_t *knn, *fwd, *nfwd, *cnt, *roff, *cursor, *rev;
    int *counter;
    double *sum;
    unsigned long long *best;
    if ((rc = s.get(&xpm, (size_t)N * g->dg_pad)) || (rc = s.get(&off, 2)) ||
        (rc = s.get(&keys, (size_t)N * (K + 1))) || (rc = s.get(&knn, (size_t)N * K)) ||
        (rc = s.get(&kd, (size_t)N * K)) || (rc = s.get(&fwd, (size_t)N * R)) ||
        (rc = s.get(&nfwd, (size_t)N)) || (rc = s.get(&cnt, (size_t)N + 1)) ||
        (rc = s.get(&roff, (size_t)N + 1)) || (rc = s.get(&cursor, (size_t)N + 1)) ||
        (rc = s.get(&rev, (size_t)N * R)) || (rc = s.get(&counter, 1)) ||
        (rc = s.get(&sum, GR_MAXDG)) || (rc = s.get(&best, 1)))
      return bail(rc);
    const int64_t h_off[2] = {0, N};
    if (cudaMemcpyAsync(off, h_off, sizeof(h_off), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "graph build"));
    // 1. K nearest other rows: one list of all rows, a dense sweep of every row
    if ((rc = launch_prefix_major(g->xg, g->dg_pad, g->dg_pad, g->dg_pad, nullptr, nullptr, nullptr,
                                  N, xpm, st)))
      return bail(rc);
    ScanArgs a{};
    a.xpm = xpm;
    a.d_pad = g->dg_pad;
    a.dims = d_g;
    a.list_off = off;
    a.qn = g->xg;
    a.ldq = g->dg_pad;
    a.nq = (int)N;
    a.counter = counter;
    a.k = K + 1;
    a.out_keys = keys;
    if ((rc = launch_scan_f32(a, st))) return bail(rc);
    knn_drop_self_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(keys, N, K, knn, kd);
    ADN_LAUNCH("knn_drop_self_kernel");
    // 2. robust prune of every candidate list
    prune_kernel<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(g->xg, g->dg_pad, d_g, knn, kd, K, N,
                                                         alpha, R, fwd, nfwd);
    ADN_LAUNCH("prune_kernel");
    // 3. offered edges grouped by target (counting sort), then the final prune
    if (cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (N + 1), st) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "graph build"));
    const int64_t ne = N * R;
    offer_count_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(fwd, ne, cnt);
    ADN_LAUNCH("offer_count_kernel");
    if ((rc = launch_scan_i32(cnt, N + 1, roff, st))) return bail(rc);
    if (cudaMemcpyAsync(cursor, roff, sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "graph build"));
    offer_fill_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(fwd, ne, R, cursor, rev);
    ADN_LAUNCH("offer_fill_kernel");
    final_prune_kernel<<<(unsigned)N, FIN_THREADS, 0, st>>>(g->xg, g->dg_pad, d_g, fwd, nfwd, roff,
                                                            rev, N, alpha, R, g->nbr, g->dev_err);
    ADN_LAUNCH("final_prune_kernel");
    // 4. entry point
    if (cudaMemsetAsync(sum, 0, sizeof(double) * GR_MAXDG, st) != cudaSuccess ||
        cudaMemsetAsync(best, 0xFF, sizeof(unsigned long long), st) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "graph build"));
    row_sum_kernel<<<1024, 64, 0, st>>>(g->xg, g->dg_pad, d_g, N, sum);
    ADN_LAUNCH("row_sum_kernel");
    entry_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(g->xg, g->dg_pad, d_g, N, sum, best);
    ADN_LAUNCH("entry_kernel");
    unsigned long long hb = 0;
    int herr = 0;
    if (cudaMemcpyAsync(&hb, best, sizeof(hb), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, g->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "graph build"));
    if (herr & ERR_HUB)
      return bail(fail(ADANNS_ERR_ARG, "a row was offered more than 4096 edges (lower R or K)"));
    g->entry = (int64_t)(hb & 0xffffffffu);
  }
  *out = g;
  return ADANNS_OK;
}

int adanns_graph_create(const float *db, int64_t N, int d, int d_g, const int32_t *graph, int R,
                        int64_t entry, int metric, void *cuda_stream, adanns_graph **out) {
  if (!out) return fail(ADANNS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!db || !graph) return fail(ADANNS_ERR_ARG, "NULL argument");
  int rc;
  if ((rc = check_graph_shape(N, d, d_g, R, metric))) return rc;
  if (entry < 0 || entry >= N) return fail(ADANNS_ERR_ARG, "entry out of range");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  adanns_graph *g = nullptr;
  if ((rc = make_shell(db, N, d, d_g, R, metric, st, &g))) return rc;
  g->entry = entry;
  if (cudaMemcpyAsync(g->nbr, graph, sizeof(int32_t) * N * R, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess) {
    free_graph(g);
    return cuda_fail(cudaGetLastError(), "graph copy");
  }
  graph_check_kernel<<<(unsigned)((N * R + 255) / 256), 256, 0, st>>>(g->nbr, N * R, N, g->dev_err);
  int bad = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&bad, g->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    free_graph(g);
    return cuda_fail(cudaGetLastError(), "graph check");
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (bad) {
    free_graph(g);
    return fail(ADANNS_ERR_ARG, "graph holds neighbour ids outside [-1, N)");
  }
  *out = g;
  return ADANNS_OK;
}

int adanns_graph_info(const adanns_graph *g, int64_t *N, int *d, int *d_g, int *R, int64_t *entry) {
  if (!g) return fail(ADANNS_ERR_ARG, "graph is NULL");
  if (N) *N = g->N;
  if (d) *d = g->d;
  if (d_g) *d_g = g->d_g;
  if (R) *R = g->R;
  if (entry) *entry = g->entry;
  return ADANNS_OK;
}

int adanns_graph_get(const adanns_graph *g, int32_t *graph, void *cuda_stream) {
  if (!g || !graph) return fail(ADANNS_ERR_ARG, "NULL argument");
  ADN_CUDA(cudaMemcpyAsync(graph, g->nbr, sizeof(int32_t) * g->N * g->R, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)cuda_stream));
  return ADANNS_OK;
}

int adanns_graph_search(const adanns_graph *g, const float *queries, int64_t B, int L, int d_s,
                        int k, int rerank_k, int64_t *out_ids, float *out_dist,
                        int64_t *out_shortlist, void *cuda_stream) {
  if (!g) return fail(ADANNS_ERR_ARG, "graph is NULL");
  if (B < 0 || B > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad batch size");
  if (B > 0 && (!queries || !out_ids || !out_dist)) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (gran_index(d_s) < 0 || d_s > g->d) return fail(ADANNS_ERR_DIM, "bad d_s");
  if (L < 1 || L > GR_MAXL) return fail(ADANNS_ERR_ARG, "need 1 <= L <= 512");
  if (k < 1 || rerank_k < k || rerank_k > L || rerank_k > 1024)
    return fail(ADANNS_ERR_ARG, "need 1 <= k <= rerank_k <= min(L, 1024)");
  if (B == 0) return ADANNS_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int dsp = pad16(d_s);
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, scratch_budget() /
                                                                  (int64_t)(dsp * 4 + 80 +
                                                                            rerank_k * 8)));
  Scratch s(st);
  float *qg, *qs;
  int64_t *sid;
  int rc;
  if ((rc = s.get(&qg, (size_t)Bc * g->dg_pad)) || (rc = s.get(&qs, (size_t)Bc * dsp)) ||
      (rc = s.get(&sid, (size_t)Bc * rerank_k)))
    return rc;
  const int cap = L + GR_MAXR;
  const size_t sm = (size_t)GS_WARPS * (2 * cap * 8 + cap + GR_MAXDG * 4);
  ADN_CUDA(ensure_smem((const void *)graph_search_kernel, sm));
  const size_t rsm = (size_t)4 * rerank_k * 8;
  ADN_CUDA(ensure_smem((const void *)graph_rerank_kernel, rsm));
  for (int64_t b0 = 0; b0 < B; b0 += Bc) {
    const int64_t nb = std::min(Bc, B - b0);
    {
      StageTimer t(ST_PREP, st);
      if ((rc = launch_prep_queries(queries + b0 * g->d, nb, g->d, g->d_g, d_s, g->metric, qg,
                                    g->dg_pad, qs, dsp, st)))
        return rc;
    }
    {
      StageTimer t(ST_SCAN, st);
      GsArgs a{};
      a.xg = g->xg;
      a.ldg = g->dg_pad;
      a.d_g = g->d_g;
      a.nbr = g->nbr;
      a.R = g->R;
      a.entry = g->entry;
      a.N = g->N;
      a.qg = qg;
      a.ldq = g->dg_pad;
      a.B = nb;
      a.L = L;
      a.kk = rerank_k;
      a.short_ids = out_shortlist ? out_shortlist + b0 * rerank_k : sid;
      graph_search_kernel<<<(unsigned)((nb + GS_WARPS - 1) / GS_WARPS), GS_WARPS * 32, sm, st>>>(a);
      ADN_LAUNCH("graph_search_kernel");
    }
    {
      StageTimer t(ST_RERANK, st);
      graph_rerank_kernel<<<(unsigned)((nb + 3) / 4), 128, rsm, st>>>(
          out_shortlist ? out_shortlist + b0 * rerank_k : sid, rerank_k, nb, qs, dsp, d_s,
          g->rows, g->d, g->metric, k, out_ids + b0 * k, out_dist + b0 * k);
      ADN_LAUNCH("graph_rerank_kernel");
    }
  }
  return ADANNS_OK;
}

void adanns_graph_free(adanns_graph *g) {
  if (!g) return;
  cudaDeviceSynchronize();
  free_graph(g);
}

}  // extern "C"
