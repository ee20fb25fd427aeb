// AdANNS-IVF search of host-resident queries with host-resident results
// (adanns_search_ivf_host).
//
// Page-locked host buffers are addressable by the GPU (over NVLink-C2C on a
// Grace-Blackwell node), so the search runs on them in place: the query-prep
// kernel reads only the first max(d_c, d_s) coordinates of each query, the
// only ones the search uses (a quarter of the rows at d_s = 512 of 2048), and
// the final kernels write the results straight into the host arrays.  There is
// no staging copy and the batch stays whole.
//
// Other host buffers go through copies: the batch is cut into slices whose
// host-to-device copy, search and device-to-host copy overlap.  The queries of slice i+1 are
// copied on a second stream while slice i is searched on the caller's stream,
// and slice i's results are copied back on that second stream while slice i+1
// is searched.  Two device buffers alternate: slice i+2's copy waits until
// slice i has been searched, and slice i+2's search waits until slice i's
// results have left.  The caller's stream waits for the last copy, so its
// completion means every result is on the host.  The search of a slice is the
// same call as on device memory; each query's results do not depend on the
// other queries of its slice.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "internal.cuh"

namespace adn {
namespace {

// the device address of page-locked host memory (null for other memory)
void *mapped(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || !a.hostPointer) return nullptr;
  return (char *)a.devicePointer + ((const char *)p - (const char *)a.hostPointer);
}

// one non-blocking copy stream per device, created on first use and kept
cudaStream_t copy_stream() {
  static std::mutex mu;
  static std::unordered_map<int, cudaStream_t> streams;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  streams[dev] = s;
  return s;
}

struct Events {
  cudaEvent_t e[16] = {};
  int n = 0;
  cudaEvent_t make() {
    if (n >= 16) return nullptr;
    cudaEvent_t x = nullptr;
    if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e[n++] = x;
  }
  ~Events() {
    for (int i = 0; i < n; ++i) cudaEventDestroy(e[i]);
  }
};

}  // namespace
}  // namespace adn

using namespace adn;

extern "C" int adanns_search_ivf_host(const adanns_index *idx, const float *queries, int64_t B,
                                      int d_c, int d_s, int nprobe, int k, int storage,
                                      int rerank_k, int64_t *out_ids, float *out_dist,
                                      int64_t slice, void *cuda_stream) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (B < 0 || B > INT32_MAX || slice < 0) return fail(ADANNS_ERR_ARG, "bad batch or slice size");
  if (B > 0 && (!queries || !out_ids || !out_dist)) return fail(ADANNS_ERR_ARG, "NULL argument");
  int rc;
  // the search's own argument checks (a call without rows launches nothing)
  if ((rc = adanns_search_ivf(idx, nullptr, 0, d_c, d_s, nprobe, k, storage, rerank_k, nullptr,
                              nullptr, nullptr, cuda_stream)))
    return rc;
  if (B == 0) return ADANNS_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  {
    const float *qm = (const float *)mapped(queries);
    int64_t *im = (int64_t *)mapped(out_ids);
    float *dm = (float *)mapped(out_dist);
    if (qm && im && dm && slice == 0)
      return adanns_search_ivf(idx, qm, B, d_c, d_s, nprobe, k, storage, rerank_k, im, dm, nullptr,
                               cuda_stream);
  }
  cudaStream_t cs = copy_stream();
  if (!cs) return fail(ADANNS_ERR_CUDA, "copy stream creation failed");
  // four slices by default: copies overlap the search of the neighbouring
  // slices, and each slice still shares its probed lists among many queries
  const int64_t S = slice > 0 ? std::min(slice, B) : std::max<int64_t>(1, (B + 3) / 4);
  const int64_t nsl = (B + S - 1) / S;
  const int d = idx->d;
  Scratch s(st);
  float *qd[2], *dd[2];
  int64_t *id[2];
  for (int b = 0; b < 2; ++b)
    if ((rc = s.get(&qd[b], (size_t)S * d)) || (rc = s.get(&id[b], (size_t)S * k)) ||
        (rc = s.get(&dd[b], (size_t)S * k)))
      return rc;
  Events ev;
  cudaEvent_t ready = ev.make();  // scratch allocated on the caller's stream
  cudaEvent_t h2d[2] = {ev.make(), ev.make()};      // slice's queries on the device
  cudaEvent_t done[2] = {ev.make(), ev.make()};     // slice searched
  cudaEvent_t d2h[2] = {ev.make(), ev.make()};      // slice's results on the host
  cudaEvent_t fin = ev.make();                      // everything queued on the copy stream
  if (!ready || !h2d[1] || !done[1] || !d2h[1] || !fin)
    return fail(ADANNS_ERR_CUDA, "event creation failed");
  ADN_CUDA(cudaEventRecord(ready, st));
  ADN_CUDA(cudaStreamWaitEvent(cs, ready, 0));
  rc = [&]() -> int {
    auto copy_in = [&](int64_t i) -> int {
      const int b = (int)(i & 1);
      const int64_t r0 = i * S, nb = std::min(S, B - r0);
      if (i >= 2) ADN_CUDA(cudaStreamWaitEvent(cs, done[b], 0));  // slice i-2 searched
      ADN_CUDA(cudaMemcpyAsync(qd[b], queries + r0 * d, sizeof(float) * nb * d,
                               cudaMemcpyHostToDevice, cs));
      ADN_CUDA(cudaEventRecord(h2d[b], cs));
      return ADANNS_OK;
    };
    if ((rc = copy_in(0))) return rc;
    for (int64_t i = 0; i < nsl; ++i) {
      const int b = (int)(i & 1);
      const int64_t r0 = i * S, nb = std::min(S, B - r0);
      // the next slice's queries travel while this one is searched
      if (i + 1 < nsl && (rc = copy_in(i + 1))) return rc;
      ADN_CUDA(cudaStreamWaitEvent(st, h2d[b], 0));
      if (i >= 2) ADN_CUDA(cudaStreamWaitEvent(st, d2h[b], 0));  // slice i-2's results left
      if ((rc = adanns_search_ivf(idx, qd[b], nb, d_c, d_s, nprobe, k, storage, rerank_k, id[b],
                                  dd[b], nullptr, st)))
        return rc;
      ADN_CUDA(cudaEventRecord(done[b], st));
      ADN_CUDA(cudaStreamWaitEvent(cs, done[b], 0));
      ADN_CUDA(cudaMemcpyAsync(out_ids + r0 * k, id[b], sizeof(int64_t) * nb * k,
                               cudaMemcpyDeviceToHost, cs));
      ADN_CUDA(cudaMemcpyAsync(out_dist + r0 * k, dd[b], sizeof(float) * nb * k,
                               cudaMemcpyDeviceToHost, cs));
      ADN_CUDA(cudaEventRecord(d2h[b], cs));
    }
    return ADANNS_OK;
  }();
  // the caller's stream (and the scratch release queued on it) waits for all
  // the copies, also when a step failed part-way
  if (cudaEventRecord(fin, cs) != cudaSuccess || cudaStreamWaitEvent(st, fin, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(cs);
  }
  return rc;
}
