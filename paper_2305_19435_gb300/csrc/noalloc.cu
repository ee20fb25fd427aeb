// AdANNS-IVF search without any device allocation.
//
// adanns_search_ivf takes its scratch (prepared queries, per-list partial
// top-k, probe inversion tables) from the CUDA stream-ordered allocator.
// Some callers cannot allocate device memory at search time: a serving
// process whose framework has already reserved the whole device memory
// budget for its own pool (a further cudaMalloc fails or fragments it),
// a latency-critical loop where an allocator call that may synchronise or
// grow a pool is not acceptable, or an embedding application whose policy
// forbids the library from touching the allocator.  For them this file
// provides the same search with its scratch in one fixed, file-scope device
// array, which every GPU that loads the library holds until the process
// exits.  Inputs and outputs are still the caller's buffers.
#include <mutex>

#include "internal.cuh"

namespace adn {
namespace {

constexpr size_t NOALLOC_BYTES = ADANNS_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array for the current device.  The name of a
// __device__ array in host code is only a host-side stand-in, so the address
// is looked up once per device (with that device current) and cached.
int scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return fail(ADANNS_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return ADANNS_OK;
}

// Bump carving of the fixed array (256-byte aligned pieces).
struct Carve {
  unsigned char *base;
  size_t used = 0;
  template <class T>
  T *take(size_t count) {
    T *p = (T *)(base + used);
    used += (count * sizeof(T) + 255) & ~(size_t)255;
    return p;
  }
};

}  // namespace
}  // namespace adn

using namespace adn;

extern "C" int adanns_search_ivf_noalloc(const adanns_index *idx, const float *queries,
                                         int64_t B, int d_c, int d_s, int nprobe, int k,
                                         int64_t *out_ids, float *out_dist, void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (B < 0 || B > INT32_MAX) return fail(ADANNS_ERR_ARG, "bad batch size");
  if (B > 0 && (!queries || !out_ids || !out_dist)) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (gran_index(d_c) < 0 || d_c > idx->d_c)
    return fail(ADANNS_ERR_DIM, "d_c must be an MR granularity <= the index's clustering prefix " +
                                    std::to_string(idx->d_c));
  if (gran_index(d_s) < 0 || d_s > idx->d)
    return fail(ADANNS_ERR_DIM, "d_s = " + std::to_string(d_s) +
                                    " is not an MR granularity within the stored dimension");
  if (nprobe < 1 || nprobe > idx->nlist) return fail(ADANNS_ERR_ARG, "need 1 <= nprobe <= nlist");
  if (k < 1 || k > 1024) return fail(ADANNS_ERR_ARG, "need 1 <= k <= 1024");
  if (B == 0) return ADANNS_OK;

  const int nlist = idx->nlist;
  const int dcp = pad16(d_c), dsp = pad16(d_s);
  const int qt = scan_query_tile(k);
  const int64_t pairs = B * nprobe;
  const int64_t max_tiles = (pairs + qt - 1) / qt + nlist;
  // measure the request against the fixed array before touching anything
  Carve need{nullptr};
  need.take<float>((size_t)B * dcp);
  need.take<float>((size_t)B * dsp);
  need.take<uint64_t>((size_t)pairs);
  need.take<uint64_t>((size_t)pairs * k);
  for (int i = 0; i < 4; ++i) need.take<int32_t>((size_t)nlist);
  need.take<int32_t>((size_t)pairs);
  need.take<int32_t>((size_t)pairs);
  for (int i = 0; i < 3; ++i) need.take<int32_t>((size_t)max_tiles);
  need.take<int>(1);
  need.take<int>(2);
  if (need.used > NOALLOC_BYTES)
    return fail(ADANNS_ERR_ARG, "request needs " + std::to_string(need.used) +
                                    " bytes of scratch; the fixed no-alloc scratch holds " +
                                    std::to_string(NOALLOC_BYTES) +
                                    " (reduce the batch, nprobe or k)");

  void *base = nullptr;
  int rc;
  if ((rc = scratch_address(&base))) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Carve c{(unsigned char *)base};
  float *qc = c.take<float>((size_t)B * dcp);
  float *qs = c.take<float>((size_t)B * dsp);
  uint64_t *ckeys = c.take<uint64_t>((size_t)pairs);
  uint64_t *pkeys = c.take<uint64_t>((size_t)pairs * k);
  int32_t *lcnt = c.take<int32_t>(nlist), *lbeg = c.take<int32_t>(nlist);
  int32_t *lfill = c.take<int32_t>(nlist), *tbeg = c.take<int32_t>(nlist);
  int32_t *pair_q = c.take<int32_t>((size_t)pairs), *pair_out = c.take<int32_t>((size_t)pairs);
  int32_t *tl = c.take<int32_t>((size_t)max_tiles), *tb = c.take<int32_t>((size_t)max_tiles);
  int32_t *tc = c.take<int32_t>((size_t)max_tiles);
  int *ntiles = c.take<int>(1);
  int *counter = c.take<int>(2);

  // the array keeps the previous call's contents: zero the work counters
  // (the list counters are zeroed inside the probe inversion)
  ADN_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st));
  if ((rc = launch_prep_queries(queries, B, idx->d, d_c, d_s, idx->metric, qc, dcp, qs, dsp, st)))
    return rc;
  ScanArgs a{};
  a.xpm = idx->cent_pm;
  a.d_pad = idx->dc_pad;  // stored centroid width; d_c <= built d_c (IVF-D)
  a.dims = d_c;
  a.list_off = idx->cent_off;
  a.qn = qc;
  a.ldq = dcp;
  a.nq = (int)B;
  a.counter = counter;
  a.k = nprobe;
  a.out_keys = ckeys;
  rc = launch_coarse(idx->centroids, idx->d_c, nlist, d_c, qc, dcp, B, nprobe, ckeys, st);
  if (rc == 1) rc = launch_scan_f32(a, st);
  if (rc) return rc;
  if ((rc = launch_invert_probes(ckeys, B, nprobe, nlist, qt, lcnt, lbeg, lfill, tbeg, pair_q,
                                 pair_out, tl, tb, tc, ntiles, nullptr, st)))
    return rc;
  ScanArgs l{};
  l.xpm = idx->xpm;
  l.d_pad = idx->d_pad;
  l.dims = d_s;
  l.list_off = idx->list_off;
  l.list_ids = idx->list_ids;
  l.mscale = idx->metric == ADANNS_METRIC_L2_PREFIXNORM
                 ? idx->invn + (int64_t)gran_index(d_s) * idx->N
                 : nullptr;
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
  if ((rc = launch_scan_f32(l, st))) return rc;
  return launch_merge(pkeys, B, nprobe, k, out_ids, out_dist, st);
}
