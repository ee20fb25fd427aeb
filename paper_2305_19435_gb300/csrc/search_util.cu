// Query preparation, probe inversion into (list, query-tile) work, and the
// cross-list top-k merge of AdANNS-IVF search (Algorithm 1 adannsInference).
#include <algorithm>
#include <cstdlib>
#include <functional>
#include <map>
#include <mutex>
#include <vector>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {

const int kGran[NGRAN] = {8, 16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 2048};

int gran_index(int m) {
  for (int i = 0; i < NGRAN; ++i)
    if (kGran[i] == m) return i;
  return -1;
}

std::atomic<long long> g_launches{0};
static thread_local std::string g_err;
void set_error(const std::string &m) { g_err = m; }
int fail(int code, const std::string &m) {
  g_err = m;
  return code;
}
int cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return ADANNS_ERR_CUDA;
}
const char *last_error() { return g_err.c_str(); }

cudaMemPool_t scratch_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = p;
  }
  return pools[dev];
}

// the largest candidate segment one query can have: the n_p longest lists,
// each padded to 8 members
int64_t max_probe_members(const adanns_index *idx, int nprobe) {
  std::vector<int64_t> len((size_t)idx->nlist);
  for (int l = 0; l < idx->nlist; ++l)
    len[(size_t)l] = (idx->h_list_off[l + 1] - idx->h_list_off[l] + 7) & ~7ll;
  std::partial_sort(len.begin(), len.begin() + nprobe, len.end(), std::greater<int64_t>());
  int64_t t = 0;
  for (int s = 0; s < nprobe; ++s) t += len[(size_t)s];
  return t;
}

// Runtime options (adanns_set_option).  The first access seeds them from the
// environment (ADANNS_FP32_STREAM, ADANNS_ADC_SELECT, ADANNS_COARSE_TC,
// ADANNS_RERANK_PRUNE, ADANNS_SCRATCH_GB); later reads are one atomic load, so
// no search call consults the environment.
namespace {
std::atomic<int64_t> g_opt[ADANNS_OPT_COUNT];
std::once_flag g_opt_once;

int64_t env_flag(const char *name, int64_t dflt) {
  const char *e = getenv(name);
  if (!e || !e[0]) return dflt;
  return e[0] == '0' ? 0 : 1;
}

void init_options() {
  std::call_once(g_opt_once, [] {
    g_opt[ADANNS_OPT_FP32_STREAM] = env_flag("ADANNS_FP32_STREAM", 1);
    g_opt[ADANNS_OPT_ADC_SELECT] = env_flag("ADANNS_ADC_SELECT", 1);
    g_opt[ADANNS_OPT_COARSE_TC] = env_flag("ADANNS_COARSE_TC", 1);
    g_opt[ADANNS_OPT_RERANK_PRUNE] = env_flag("ADANNS_RERANK_PRUNE", 1);
    const char *e = getenv("ADANNS_SCRATCH_GB");
    double gb = e ? atof(e) : 12.0;
    if (!(gb > 0.0)) gb = 12.0;
    g_opt[ADANNS_OPT_SCRATCH_BYTES] = (int64_t)(gb * (double)(1ll << 30));
    g_opt[ADANNS_OPT_WAIT_LIMIT_NS] = 2000000000ll;
    g_opt[ADANNS_OPT_TEST_SKIP_LOAD] = -1;
    g_opt[ADANNS_OPT_SCAN_FILTER] = 0;
    g_opt[ADANNS_OPT_NARROW_SCAN] = 1;
  });
}
}  // namespace

int64_t option(int o) {
  init_options();
  return g_opt[o].load(std::memory_order_relaxed);
}

int64_t take_option(int o, int64_t reset) {
  init_options();
  return g_opt[o].exchange(reset);
}

int set_option(int o, int64_t v) {
  init_options();
  if (o < 0 || o >= ADANNS_OPT_COUNT) return fail(ADANNS_ERR_ARG, "unknown option");
  switch (o) {
    case ADANNS_OPT_FP32_STREAM:
    case ADANNS_OPT_ADC_SELECT:
    case ADANNS_OPT_COARSE_TC:
    case ADANNS_OPT_RERANK_PRUNE:
    case ADANNS_OPT_SCAN_FILTER:
      if (v != 0 && v != 1) return fail(ADANNS_ERR_ARG, "this option takes 0 or 1");
      break;
    case ADANNS_OPT_NARROW_SCAN:
      if (v < 0 || v > 2) return fail(ADANNS_ERR_ARG, "this option takes 0, 1 or 2");
      break;
    case ADANNS_OPT_SCRATCH_BYTES:
      if (v < (1ll << 20)) return fail(ADANNS_ERR_ARG, "scratch budget below 1 MiB");
      break;
    case ADANNS_OPT_WAIT_LIMIT_NS:
      if (v < 100000 || v > 60000000000ll)
        return fail(ADANNS_ERR_ARG, "wait limit must be within [1e5, 6e10] ns");
      break;
    case ADANNS_OPT_TEST_SKIP_LOAD:
      if (v < -1 || v > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad skip index");
      break;
  }
  g_opt[o].store(v);
  return ADANNS_OK;
}

int64_t scratch_budget() { return option(ADANNS_OPT_SCRATCH_BYTES); }

cudaError_t ensure_smem(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  auto key = std::make_pair(dev, fn);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

int num_sms() {
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (!sms[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 148;
  }
  return sms[dev];
}

// ---------------------------------------------------------------- queries
// Per query (one warp): inverse prefix norms at dims_a and dims_b (FP32 sums
// of squares, lane-strided then a shuffle tree) and the two scaled, zero
// padded copies q * nu_a (rows of lda) and q * nu_b (rows of ldb).
__global__ void prep_queries_kernel(const float *__restrict__ q, int64_t B, int ld, int da,
                                    int db0, int metric, float *__restrict__ qa, int lda,
                                    float *__restrict__ qb, int ldb,
                                    const int32_t *__restrict__ dbq,
                                    const int32_t *__restrict__ rows) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= B) return;
  const int db = dbq ? dbq[row] : db0;
  const float *src = q + (rows ? (int64_t)rows[row] : row) * ld;
  float sa = 0.f, sb = 0.f;
  const int dm = max(da, db);
  for (int j = lane; j < dm; j += 32) {
    const float v = src[j];
    if (j < da) sa = fmaf(v, v, sa);
    if (j < db) sb = fmaf(v, v, sb);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  float na = 1.f, nb = 1.f;
  if (metric == ADANNS_METRIC_L2_PREFIXNORM) {
    na = sa > 0.f ? 1.f / sqrtf(sa) : 0.f;
    nb = sb > 0.f ? 1.f / sqrtf(sb) : 0.f;
  }
  if (qa)
    for (int j = lane; j < lda; j += 32) qa[row * lda + j] = j < da ? src[j] * na : 0.f;
  if (qb)
    for (int j = lane; j < ldb; j += 32) qb[row * ldb + j] = j < db ? src[j] * nb : 0.f;
}

// The same for rows of at most 2,048 used coordinates, 16-byte aligned: each
// lane loads its share of the row prefix (up to 16 float4) once, all loads in
// flight together, and both copies are written from registers.  Query rows in
// host memory read over the host link are read exactly once this way.
template <int PV>  // float4 per lane: PV x 4 x 32 coordinates (4: 512, 8: 1,024, 16: 2,048)
__global__ void __launch_bounds__(256) prep_queries_v4_kernel(
    const float *__restrict__ q, int64_t B, int ld, int da, int db0, int metric,
    float *__restrict__ qa, int lda, float *__restrict__ qb, int ldb,
    const int32_t *__restrict__ dbq, const int32_t *__restrict__ rows) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= B) return;
  const int db = dbq ? dbq[row] : db0;
  const float4 *src = (const float4 *)(q + (rows ? (int64_t)rows[row] : row) * ld);
  const int dm = max(da, db), nv = (dm + 3) >> 2;
  float4 v[PV];
#pragma unroll
  for (int t = 0; t < PV; ++t) {
    const int c = lane + 32 * t;
    v[t] = c < nv ? src[c] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float sa = 0.f, sb = 0.f;
#pragma unroll
  for (int t = 0; t < PV; ++t) {
    const int j = 4 * (lane + 32 * t);
    const float e[4] = {v[t].x, v[t].y, v[t].z, v[t].w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (j + u < da) sa = fmaf(e[u], e[u], sa);
      if (j + u < db) sb = fmaf(e[u], e[u], sb);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  float na = 1.f, nb = 1.f;
  if (metric == ADANNS_METRIC_L2_PREFIXNORM) {
    na = sa > 0.f ? 1.f / sqrtf(sa) : 0.f;
    nb = sb > 0.f ? 1.f / sqrtf(sb) : 0.f;
  }
  auto put = [&](float *dst, int ldd, int dd, float nrm) {
    if (!dst) return;
#pragma unroll
    for (int t = 0; t < PV; ++t) {
      const int j = 4 * (lane + 32 * t);
      if (j >= ldd) break;
      const float4 x = v[t];
      const float4 y = make_float4(j < dd ? x.x * nrm : 0.f, j + 1 < dd ? x.y * nrm : 0.f,
                                   j + 2 < dd ? x.z * nrm : 0.f, j + 3 < dd ? x.w * nrm : 0.f);
      *(float4 *)(dst + row * ldd + j) = y;
    }
    for (int j = 4 * (lane + 32 * PV); j < ldd; j += 128)  // padding past the loaded prefix
      *(float4 *)(dst + row * ldd + j) = make_float4(0.f, 0.f, 0.f, 0.f);
  };
  put(qa, lda, da, na);
  put(qb, ldb, db, nb);
}

int launch_prep_queries(const float *q, int64_t B, int ld, int da, int db, int metric, float *qa,
                        int lda, float *qb, int ldb, cudaStream_t st, const int32_t *dbq,
                        const int32_t *rows) {
  if (B <= 0) return ADANNS_OK;
  const int wpb = 8;
  // per-query d_s up to db (the batch's largest); lda / ldb multiples of 16
  if (std::max(da, db) <= 2048 && (ld & 3) == 0 && ((uintptr_t)q & 15) == 0 &&
      (lda & 3) == 0 && (ldb & 3) == 0) {
    const int dm = std::max(da, db);
    const dim3 grid((unsigned)((B + wpb - 1) / wpb));
    if (dm <= 512)
      prep_queries_v4_kernel<4><<<grid, wpb * 32, 0, st>>>(q, B, ld, da, db, metric, qa, lda, qb,
                                                           ldb, dbq, rows);
    else if (dm <= 1024)
      prep_queries_v4_kernel<8><<<grid, wpb * 32, 0, st>>>(q, B, ld, da, db, metric, qa, lda, qb,
                                                           ldb, dbq, rows);
    else
      prep_queries_v4_kernel<16><<<grid, wpb * 32, 0, st>>>(q, B, ld, da, db, metric, qa, lda, qb,
                                                            ldb, dbq, rows);
    ADN_LAUNCH("prep_queries_v4_kernel");
    return ADANNS_OK;
  }
  prep_queries_kernel<<<(unsigned)((B + wpb - 1) / wpb), wpb * 32, 0, st>>>(
      q, B, ld, da, db, metric, qa, lda, qb, ldb, dbq, rows);
  ADN_LAUNCH("prep_queries_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- keys -> results
__global__ void keys_to_result_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                      int64_t *__restrict__ ids, int32_t *__restrict__ ids32,
                                      float *__restrict__ dist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  const bool pad = k == KEY_MAX;
  if (ids) ids[i] = pad ? -1 : (int64_t)(uint32_t)(k & 0xffffffffu);
  if (ids32) ids32[i] = pad ? -1 : (int32_t)(uint32_t)(k & 0xffffffffu);
  if (dist) dist[i] = pad ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(k >> 32));
}

int launch_keys_to_result(const uint64_t *keys, int64_t rows, int k, int64_t *ids, int32_t *ids32,
                          float *dist, cudaStream_t st) {
  const int64_t n = rows * k;
  if (n <= 0) return ADANNS_OK;
  keys_to_result_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, n, ids, ids32, dist);
  ADN_LAUNCH("keys_to_result_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- probe inversion
// Pairs (query, probe slot) over slots [s0, s0 + ns) of each query's nprobe:
// item i is pair e = (i / ns) * nprobe + s0 + i % ns.
__device__ __forceinline__ int64_t slot_pair(int64_t i, int nprobe, int s0, int ns) {
  return ns == nprobe ? i : (i / ns) * nprobe + s0 + i % ns;
}

__global__ void probe_count_kernel(const uint64_t *__restrict__ ckeys, int64_t n, int nprobe,
                                   int s0, int ns, int32_t *__restrict__ lcnt,
                                   int32_t *__restrict__ probes_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = slot_pair(i, nprobe, s0, ns);
  const int l = probe_list(ckeys[e]);
  if (probes_out) probes_out[e] = l;
  if (l >= 0) atomicAdd(&lcnt[l], 1);
}

// single CTA: lbeg = exclusive scan of lcnt; per-list tile counts and their scan
__global__ void probe_scan_kernel(const int32_t *__restrict__ lcnt, int nlist, int qt,
                                  int32_t *__restrict__ lbeg, int32_t *__restrict__ tbeg,
                                  int *__restrict__ ntiles) {
  __shared__ int32_t s_a[1024], s_b[1024];
  __shared__ int32_t carry_a, carry_b;
  if (threadIdx.x == 0) carry_a = carry_b = 0;
  __syncthreads();
  for (int base = 0; base < nlist; base += 1024) {
    const int l = base + threadIdx.x;
    const int c = l < nlist ? lcnt[l] : 0;
    const int t = (c + qt - 1) / qt;
    s_a[threadIdx.x] = c;
    s_b[threadIdx.x] = t;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int va = 0, vb = 0;
      if ((int)threadIdx.x >= o) { va = s_a[threadIdx.x - o]; vb = s_b[threadIdx.x - o]; }
      __syncthreads();
      s_a[threadIdx.x] += va;
      s_b[threadIdx.x] += vb;
      __syncthreads();
    }
    if (l < nlist) {
      lbeg[l] = carry_a + s_a[threadIdx.x] - c;
      tbeg[l] = carry_b + s_b[threadIdx.x] - t;
    }
    __syncthreads();
    if (threadIdx.x == 1023) { carry_a += s_a[1023]; carry_b += s_b[1023]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ntiles = carry_b;
}

__global__ void probe_fill_kernel(const uint64_t *__restrict__ ckeys, int64_t n, int nprobe,
                                  int s0, int ns, const int32_t *__restrict__ lbeg,
                                  int32_t *__restrict__ lfill, int32_t *__restrict__ pair_q,
                                  int32_t *__restrict__ pair_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = slot_pair(i, nprobe, s0, ns);
  const int l = probe_list(ckeys[e]);
  if (l < 0) return;  // a masked slot has no pair
  const int pos = lbeg[l] + atomicAdd(&lfill[l], 1);
  pair_q[pos] = (int32_t)(e / nprobe);
  pair_out[pos] = (int32_t)e;
}

// Block-aggregated variants for lists of at most PB_MAXL (the common case):
// a block takes PB_ITEMS consecutive pairs, counts them per list in shared
// memory and touches each list's global counter once, so the global atomics
// (which contend when many queries probe one list) drop by about the number of
// the block's pairs per list.  Fill reserves one range per (block, list) and
// places the block's pairs in it in item order.
constexpr int PB_THREADS = 256;
constexpr int PB_ITEMS = 4096;
constexpr int PB_MAXL = 8192;

__global__ void __launch_bounds__(PB_THREADS) probe_count_block_kernel(
    const uint64_t *__restrict__ ckeys, int64_t n, int nprobe, int s0, int ns, int nlist,
    int32_t *__restrict__ lcnt, int32_t *__restrict__ probes_out) {
  extern __shared__ int s_hist[];  // [nlist]
  for (int b = threadIdx.x; b < nlist; b += PB_THREADS) s_hist[b] = 0;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * PB_ITEMS;
  for (int j = threadIdx.x; j < PB_ITEMS; j += PB_THREADS) {
    const int64_t i = i0 + j;
    if (i >= n) break;
    const int64_t e = slot_pair(i, nprobe, s0, ns);
    const int l = probe_list(ckeys[e]);
    if (probes_out) probes_out[e] = l;
    if (l >= 0) atomicAdd(&s_hist[l], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nlist; b += PB_THREADS)
    if (s_hist[b]) atomicAdd(&lcnt[b], s_hist[b]);
}

__global__ void __launch_bounds__(PB_THREADS) probe_fill_block_kernel(
    const uint64_t *__restrict__ ckeys, int64_t n, int nprobe, int s0, int ns, int nlist,
    const int32_t *__restrict__ lbeg, int32_t *__restrict__ lfill, int32_t *__restrict__ pair_q,
    int32_t *__restrict__ pair_out) {
  extern __shared__ int s_hist[];  // [nlist] counts, then [nlist] positions
  int *s_pos = s_hist + nlist;
  for (int b = threadIdx.x; b < nlist; b += PB_THREADS) s_hist[b] = 0;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * PB_ITEMS;
  for (int j = threadIdx.x; j < PB_ITEMS; j += PB_THREADS) {
    const int64_t i = i0 + j;
    if (i >= n) break;
    const int l = probe_list(ckeys[slot_pair(i, nprobe, s0, ns)]);
    if (l >= 0) atomicAdd(&s_hist[l], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nlist; b += PB_THREADS) {
    const int c = s_hist[b];
    s_pos[b] = c ? lbeg[b] + atomicAdd(&lfill[b], c) : 0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < PB_ITEMS; j += PB_THREADS) {
    const int64_t i = i0 + j;
    if (i >= n) break;
    const int64_t e = slot_pair(i, nprobe, s0, ns);
    const int l = probe_list(ckeys[e]);
    if (l < 0) continue;  // a masked slot has no pair
    const int pos = atomicAdd(&s_pos[l], 1);
    pair_q[pos] = (int32_t)(e / nprobe);
    pair_out[pos] = (int32_t)e;
  }
}

__global__ void probe_tiles_kernel(const int32_t *__restrict__ lcnt,
                                   const int32_t *__restrict__ lbeg,
                                   const int32_t *__restrict__ tbeg, int nlist, int qt,
                                   int32_t *__restrict__ tile_list, int32_t *__restrict__ tile_beg,
                                   int32_t *__restrict__ tile_cnt) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlist) return;
  const int c = lcnt[l];
  const int nt = (c + qt - 1) / qt;
  for (int t = 0; t < nt; ++t) {
    const int idx = tbeg[l] + t;
    tile_list[idx] = l;
    tile_beg[idx] = lbeg[l] + t * qt;
    tile_cnt[idx] = min(qt, c - t * qt);
  }
}

int launch_invert_probes(const uint64_t *ckeys, int64_t B, int nprobe, int nlist, int qt,
                         int32_t *lcnt, int32_t *lbeg, int32_t *lfill, int32_t *tbeg,
                         int32_t *pair_q, int32_t *pair_out, int32_t *tile_list,
                         int32_t *tile_beg, int32_t *tile_cnt, int *ntiles, int32_t *probes_out,
                         cudaStream_t st) {
  return launch_invert_probe_slots(ckeys, B, nprobe, 0, nprobe, nlist, qt, lcnt, lbeg, lfill, tbeg,
                                   pair_q, pair_out, tile_list, tile_beg, tile_cnt, ntiles,
                                   probes_out, st);
}

int launch_invert_probe_slots(const uint64_t *ckeys, int64_t B, int nprobe, int s0, int ns,
                              int nlist, int qt, int32_t *lcnt, int32_t *lbeg, int32_t *lfill,
                              int32_t *tbeg, int32_t *pair_q, int32_t *pair_out,
                              int32_t *tile_list, int32_t *tile_beg, int32_t *tile_cnt,
                              int *ntiles, int32_t *probes_out, cudaStream_t st) {
  const int64_t n = B * ns;
  ADN_CUDA(cudaMemsetAsync(lcnt, 0, sizeof(int32_t) * nlist, st));
  ADN_CUDA(cudaMemsetAsync(lfill, 0, sizeof(int32_t) * nlist, st));
  const unsigned g = (unsigned)((std::max<int64_t>(n, 1) + 255) / 256);
  // block-aggregated counting when many pairs share each list
  const bool blocked = nlist <= PB_MAXL && n >= (int64_t)4 * nlist;
  const unsigned gb = (unsigned)((std::max<int64_t>(n, 1) + PB_ITEMS - 1) / PB_ITEMS);
  if (blocked) {
    const size_t sm = sizeof(int) * nlist;
    ADN_CUDA(ensure_smem((const void *)probe_count_block_kernel, sm));
    probe_count_block_kernel<<<gb, PB_THREADS, sm, st>>>(ckeys, n, nprobe, s0, ns, nlist, lcnt,
                                                         probes_out);
    ADN_LAUNCH("probe_count_block_kernel");
  } else {
    probe_count_kernel<<<g, 256, 0, st>>>(ckeys, n, nprobe, s0, ns, lcnt, probes_out);
    ADN_LAUNCH("probe_count_kernel");
  }
  probe_scan_kernel<<<1, 1024, 0, st>>>(lcnt, nlist, qt, lbeg, tbeg, ntiles);
  ADN_LAUNCH("probe_scan_kernel");
  if (blocked) {
    const size_t sm = sizeof(int) * 2 * nlist;
    ADN_CUDA(ensure_smem((const void *)probe_fill_block_kernel, sm));
    probe_fill_block_kernel<<<gb, PB_THREADS, sm, st>>>(ckeys, n, nprobe, s0, ns, nlist, lbeg,
                                                        lfill, pair_q, pair_out);
    ADN_LAUNCH("probe_fill_block_kernel");
  } else {
    probe_fill_kernel<<<g, 256, 0, st>>>(ckeys, n, nprobe, s0, ns, lbeg, lfill, pair_q, pair_out);
    ADN_LAUNCH("probe_fill_kernel");
  }
  probe_tiles_kernel<<<(nlist + 255) / 256, 256, 0, st>>>(lcnt, lbeg, tbeg, nlist, qt, tile_list,
                                                          tile_beg, tile_cnt);
  ADN_LAUNCH("probe_tiles_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- per-query budgets
__global__ void mask_probes_kernel(uint64_t *__restrict__ ckeys, int64_t n, int nprobe,
                                   const int32_t *__restrict__ np) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  if ((int)(e % nprobe) >= np[e / nprobe]) ckeys[e] = PROBE_NONE;
}

int launch_mask_probes(uint64_t *ckeys, int64_t B, int nprobe, const int32_t *np,
                       cudaStream_t st) {
  const int64_t n = B * nprobe;
  if (n <= 0 || !np) return ADANNS_OK;
  mask_probes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ckeys, n, nprobe, np);
  ADN_LAUNCH("mask_probes_kernel");
  return ADANNS_OK;
}

__global__ void pad_rows_kernel(int64_t *__restrict__ ids, float *__restrict__ dist, int64_t n,
                                int k_max, const int32_t *__restrict__ k) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if ((int)(i % k_max) >= k[i / k_max]) {
    ids[i] = -1;
    dist[i] = __int_as_float(0x7f800000);
  }
}

int launch_pad_rows(int64_t *ids, float *dist, int64_t B, int k_max, const int32_t *k,
                    cudaStream_t st) {
  const int64_t n = B * k_max;
  if (n <= 0 || !k) return ADANNS_OK;
  pad_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ids, dist, n, k_max, k);
  ADN_LAUNCH("pad_rows_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- merge
// Per query (one warp): the nprobe sorted per-list top-k runs -> the k best.
// tau starts at the smallest k-th key over the runs, an upper bound of the
// final k-th key, so only keys <= tau are buffered; the buffer is sorted and
// trimmed to k whenever it fills.  Per-query budgets (m.ckeys non-null): run r
// belongs to probe slot r / m.nsplit, and runs of masked slots (PROBE_NONE,
// never scanned) are skipped; m.kq: the query keeps its first kq[q] results
// and pads the rest; m.orow: the query's output row.
constexpr int MERGE_WPB = 4;

__global__ void merge_kernel(const uint64_t *__restrict__ pkeys, int64_t B, int nprobe, int k,
                             int cap, int64_t *__restrict__ out_ids,
                             float *__restrict__ out_dist, MergeMask m) {
  extern __shared__ uint64_t msmem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t qi = (int64_t)blockIdx.x * MERGE_WPB + warp;
  if (qi >= B) return;
  uint64_t *buf = msmem + (size_t)warp * cap;
  const uint64_t *src = pkeys + qi * (int64_t)nprobe * k;
  const int nslot = m.ckeys ? nprobe / m.nsplit : 0;
  auto masked = [&](int run) -> bool {
    return m.ckeys && m.ckeys[qi * nslot + run / m.nsplit] == PROBE_NONE;
  };
  uint64_t tau = KEY_MAX;
  for (int s = lane; s < nprobe; s += 32) {
    const uint64_t v = masked(s) ? KEY_MAX : src[(int64_t)s * k + k - 1];
    tau = v < tau ? v : tau;
  }
  tau = warp_min_u64(tau);
  int n = 0;
  const int total = nprobe * k;
  for (int base = 0; base < total; base += 32) {
    const int i = base + lane;
    const uint64_t key = i < total && !masked(i / k) ? src[i] : KEY_MAX;
    const bool take = key != KEY_MAX && key <= tau;
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (take) buf[n + __popc(m & lanemask_lt())] = key;
    n += __popc(m);
    if (n > cap - 32) {
      __syncwarp();
      warp_sort(buf, n);
      if (n > k) n = k;
      if (n == k) {
        const uint64_t kth = buf[k - 1];
        tau = kth < tau ? kth : tau;
      }
      __syncwarp();
    }
  }
  __syncwarp();
  warp_sort(buf, n);
  if (n > k) n = k;
  if (m.kq && n > m.kq[qi]) n = m.kq[qi];
  const int64_t orow = m.orow ? (int64_t)m.orow[qi] : qi;
  for (int r = lane; r < k; r += 32) {
    const int64_t o = orow * k + r;
    if (r < n) {
      const uint64_t key = buf[r];
      out_ids[o] = (int64_t)(uint32_t)(key & 0xffffffffu);
      out_dist[o] = __uint_as_float((uint32_t)(key >> 32));
    } else {
      out_ids[o] = -1;
      out_dist[o] = __int_as_float(0x7f800000);
    }
  }
}

int launch_merge(const uint64_t *pkeys, int64_t B, int nprobe, int k, int64_t *out_ids,
                 float *out_dist, cudaStream_t st, const MergeMask &mm) {
  if (B <= 0) return ADANNS_OK;
  int kp = 1;
  while (kp < k) kp <<= 1;
  int cap = 2 * kp;
  if (cap < kp + 32) cap = kp + 32;
  const size_t smem = (size_t)MERGE_WPB * cap * 8;
  cudaError_t e = ensure_smem((const void *)merge_kernel, smem);
  if (e != cudaSuccess) return cuda_fail(e, "merge attribute");
  merge_kernel<<<(unsigned)((B + MERGE_WPB - 1) / MERGE_WPB), MERGE_WPB * 32, smem, st>>>(
      pkeys, B, nprobe, k, cap, out_ids, out_dist, mm);
  ADN_LAUNCH("merge_kernel");
  return ADANNS_OK;
}

}  // namespace adn
