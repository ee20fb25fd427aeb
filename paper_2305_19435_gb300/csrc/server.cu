// Continuous-batching search server (adanns_server_*): the serving loop of the
// compute-aware elastic search of Sec. 5 ("Compute-aware Elastic Search
// During Inference"), where every request carries its own compute budget
// (d_c, d_s, nprobe, k, tier) over indices that stay resident.
//
// Requests are host query batches submitted at any time.  A worker thread
// keeps them in arrival order and, whenever one of the server's CUDA streams
// is free, packs the oldest request with later requests of the same index whose
// budgets can share one pass of the search (below) into one batch of at most
// max_batch rows, admits the batch only if
// its scratch estimate fits the memory budget next to the batches in flight
// (a batch is always admitted when nothing is in flight), and launches it on
// that stream: the rows are staged in pinned memory, copied to the device,
// searched, and the results copied back, followed by an event.  Batches on
// different streams overlap on the device; the worker polls their events and
// hands each request its rows.  Callers collect results with
// adanns_server_poll.
//
// Budgets that share a pass (adanns_search_ivf_budgets /
// adanns_search_ivfopq_budgets): with the FP32 tier, any d_s, nprobe (<= 256)
// and k at one d_c; with a low-precision tier, any nprobe and k at one d_c,
// d_s and rerank_k; IVF-OPQ, any nprobe (<= 256) and k at one d_c and
// rerank_k.  A batch of one budget runs the plain search call, a mixed one the
// per-query-budget call.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace adn {
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  int64_t ticket = 0;
  int slot = 0;  // index slot
  adanns_budget b{};
  int64_t n = 0;
  std::vector<float> q;  // host copy of the rows
  std::vector<int64_t> ids;
  std::vector<float> dist;
  int status = 1;  // ADANNS_PENDING until finished
  std::string msg;
  double t_arrive = 0.0, t_done = 0.0;
};

// A grow-only device or pinned host buffer.
struct Buf {
  void *p = nullptr;
  size_t cap = 0;
  bool host = false;
  int need(size_t bytes) {
    if (bytes <= cap) return ADANNS_OK;
    if (p) host ? cudaFreeHost(p) : cudaFree(p);
    p = nullptr;
    cap = 0;
    const cudaError_t e = host ? cudaMallocHost(&p, bytes) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(ADANNS_ERR_OOM, "server buffer allocation of " + std::to_string(bytes) +
                                      " bytes failed");
    }
    cap = bytes;
    return ADANNS_OK;
  }
  ~Buf() {
    if (p) host ? cudaFreeHost(p) : cudaFree(p);
  }
};

struct Lane {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<std::shared_ptr<Request>> reqs;
  int64_t bytes = 0;
  int kstride = 0;  // result columns per row of the batch (its largest k)
  Buf qh{nullptr, 0, true}, ih{nullptr, 0, true}, dh{nullptr, 0, true};
  Buf qd, id, dd;
};

bool same_budget(const adanns_budget &a, const adanns_budget &b) {
  return a.method == b.method && a.d_c == b.d_c && a.d_s == b.d_s && a.nprobe == b.nprobe &&
         a.k == b.k && a.storage == b.storage && a.rerank_k == b.rerank_k;
}

// whether requests with budgets a and b can run in one pass of the search
bool shareable(const adanns_budget &a, const adanns_budget &b) {
  if (same_budget(a, b)) return true;
  if (a.method != b.method || a.d_c != b.d_c || a.rerank_k != b.rerank_k) return false;
  if (a.method == ADANNS_METHOD_IVFOPQ) return a.nprobe <= 256 && b.nprobe <= 256;
  if (a.method != ADANNS_METHOD_IVF || a.storage != b.storage) return false;
  if (a.storage == ADANNS_STORE_F32) return a.nprobe <= 256 && b.nprobe <= 256;
  return a.d_s == b.d_s;
}

}  // namespace
}  // namespace adn

using namespace adn;

struct adanns_server {
  std::vector<const adanns_index *> indices;
  int device = 0;
  int64_t max_batch = 0, mem_budget = 0;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<int64_t, std::shared_ptr<Request>> live;
  int64_t next_ticket = 1;
  int64_t inflight = 0;
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> lat_ms;
  int64_t batches = 0, batch_requests = 0, queries = 0, max_inflight = 0;
  double t_first = 0.0, t_last = 0.0;

  void finish(Lane &L);
  bool launch_one(Lane &L);
  void loop();
};

// scatter a finished batch's rows to its requests
void adanns_server::finish(Lane &L) {
  const cudaError_t e = cudaEventSynchronize(L.done);
  const double t = now_ms();
  int64_t off = 0;
  std::lock_guard<std::mutex> g(mu);
  for (auto &r : L.reqs) {
    if (e != cudaSuccess) {
      r->status = ADANNS_ERR_CUDA;
      r->msg = std::string("batch failed: ") + cudaGetErrorString(e);
    } else {
      const int k = r->b.k, ks = L.kstride;  // the request's first k of each row
      r->ids.resize((size_t)(r->n * k));
      r->dist.resize((size_t)(r->n * k));
      for (int64_t i = 0; i < r->n; ++i) {
        memcpy(r->ids.data() + i * k, (const int64_t *)L.ih.p + (off + i) * ks, sizeof(int64_t) * k);
        memcpy(r->dist.data() + i * k, (const float *)L.dh.p + (off + i) * ks, sizeof(float) * k);
      }
      r->status = ADANNS_OK;
      lat_ms.push_back(t - r->t_arrive);
      queries += r->n;
    }
    r->t_done = t;
    t_last = std::max(t_last, t);
    off += r->n;
  }
  L.reqs.clear();
  L.busy = false;
  inflight -= L.bytes;
  L.bytes = 0;
  cv_done.notify_all();
}

// take the next batch (if admitted) and launch it on lane L; false if nothing was launched
bool adanns_server::launch_one(Lane &L) {
  std::vector<std::shared_ptr<Request>> batch;
  int64_t rows = 0, bytes = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    if (pending.empty()) return false;
    const auto head = pending.front();
    std::deque<std::shared_ptr<Request>> keep;
    for (auto &r : pending) {
      if (r->slot == head->slot && shareable(r->b, head->b) &&
          (batch.empty() || rows + r->n <= max_batch)) {
        batch.push_back(r);
        rows += r->n;
      } else {
        keep.push_back(r);
      }
    }
    const adanns_index *idx = indices[(size_t)head->slot];
    adanns_budget b = head->b;  // the batch's largest d_s, nprobe and k
    bool mixed = false;
    for (auto &r : batch) {
      mixed = mixed || !same_budget(r->b, b);
      b.d_s = std::max(b.d_s, r->b.d_s);
      b.nprobe = std::max(b.nprobe, r->b.nprobe);
      b.k = std::max(b.k, r->b.k);
    }
    if (b.method == ADANNS_METHOD_IVFOPQ)
      bytes = rows * (int64_t)(b.nprobe * 64 + b.k * 12 + idx->d * 4) + (64ll << 20);
    else if (mixed && b.storage == ADANNS_STORE_F32)
      bytes = stream_scratch_bytes(idx, rows, b.d_c, b.d_s, b.nprobe, b.k);
    else
      bytes = adanns_search_scratch_bytes(idx, rows, b.d_c, b.d_s, b.nprobe, b.k, b.storage,
                                          b.rerank_k);
    if (bytes < 0) bytes = 0;
    bytes += rows * (int64_t)(idx->d * 4 + b.k * 12 + (mixed ? 16 : 0));
    const bool any_busy = std::any_of(lanes.begin(), lanes.end(),
                                      [](const std::unique_ptr<Lane> &x) { return x->busy; });
    if (any_busy && inflight + bytes > mem_budget) return false;  // wait for memory
    pending.swap(keep);
    inflight += bytes;
    max_inflight = std::max(max_inflight, inflight);
    batches += 1;
    batch_requests += (int64_t)batch.size();
  }
  const adanns_index *idx = indices[(size_t)batch[0]->slot];
  adanns_budget b = batch[0]->b;
  bool mixed = false;
  for (auto &r : batch) {
    mixed = mixed || !same_budget(r->b, b);
    b.k = std::max(b.k, r->b.k);
  }
  const int d = idx->d, k = b.k;
  int rc = ADANNS_OK;
  std::string msg;
  if ((rc = L.qh.need(sizeof(float) * rows * d)) || (rc = L.ih.need(sizeof(int64_t) * rows * k)) ||
      (rc = L.dh.need(sizeof(float) * rows * k)) || (rc = L.qd.need(sizeof(float) * rows * d)) ||
      (rc = L.id.need(sizeof(int64_t) * rows * k)) || (rc = L.dd.need(sizeof(float) * rows * k))) {
    msg = adanns_last_error();
  } else {
    int64_t off = 0;
    for (auto &r : batch) {
      memcpy((float *)L.qh.p + off * d, r->q.data(), sizeof(float) * r->n * d);
      off += r->n;
    }
    cudaError_t e = cudaMemcpyAsync(L.qd.p, L.qh.p, sizeof(float) * rows * d,
                                    cudaMemcpyHostToDevice, L.st);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "server query copy");
    } else if (mixed) {
      std::vector<int32_t> ds((size_t)rows), np((size_t)rows), kq((size_t)rows);
      int64_t o = 0;
      for (auto &r : batch)
        for (int64_t i = 0; i < r->n; ++i, ++o) {
          ds[(size_t)o] = r->b.d_s;
          np[(size_t)o] = r->b.nprobe;
          kq[(size_t)o] = r->b.k;
        }
      rc = b.method == ADANNS_METHOD_IVFOPQ
               ? adanns_search_ivfopq_budgets(idx, (const float *)L.qd.p, rows, b.d_c, np.data(),
                                              kq.data(), k, b.rerank_k, (int64_t *)L.id.p,
                                              (float *)L.dd.p, L.st)
               : adanns_search_ivf_budgets(idx, (const float *)L.qd.p, rows, b.d_c, ds.data(),
                                           np.data(), kq.data(), k, b.storage, b.rerank_k,
                                           (int64_t *)L.id.p, (float *)L.dd.p, L.st);
    } else if (b.method == ADANNS_METHOD_IVFOPQ) {
      rc = adanns_search_ivfopq(idx, (const float *)L.qd.p, rows, b.d_c, b.nprobe, k, b.rerank_k,
                                (int64_t *)L.id.p, (float *)L.dd.p, nullptr, L.st);
    } else {
      rc = adanns_search_ivf(idx, (const float *)L.qd.p, rows, b.d_c, b.d_s, b.nprobe, k,
                             b.storage, b.rerank_k, (int64_t *)L.id.p, (float *)L.dd.p, nullptr,
                             L.st);
    }
    if (rc == ADANNS_OK) {
      if ((e = cudaMemcpyAsync(L.ih.p, L.id.p, sizeof(int64_t) * rows * k, cudaMemcpyDeviceToHost,
                               L.st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(L.dh.p, L.dd.p, sizeof(float) * rows * k, cudaMemcpyDeviceToHost,
                               L.st)) != cudaSuccess ||
          (e = cudaEventRecord(L.done, L.st)) != cudaSuccess)
        rc = cuda_fail(e, "server result copy");
    }
    if (rc) msg = adanns_last_error();
  }
  if (rc) {  // the batch never reached the device: every request reports the error
    std::lock_guard<std::mutex> g(mu);
    const double t = now_ms();
    for (auto &r : batch) {
      r->status = rc;
      r->msg = msg;
      r->t_done = t;
    }
    inflight -= bytes;
    cv_done.notify_all();
    return true;
  }
  L.reqs = std::move(batch);
  L.bytes = bytes;
  L.kstride = k;
  L.busy = true;
  return true;
}

void adanns_server::loop() {
  cudaSetDevice(device);
  for (;;) {
    bool progressed = false;
    for (auto &lp : lanes) {
      Lane &L = *lp;
      if (L.busy && cudaEventQuery(L.done) != cudaErrorNotReady) {
        cudaGetLastError();
        finish(L);
        progressed = true;
      }
    }
    for (auto &lp : lanes)
      if (!lp->busy && launch_one(*lp)) progressed = true;
    std::unique_lock<std::mutex> g(mu);
    const bool busy = std::any_of(lanes.begin(), lanes.end(),
                                  [](const std::unique_ptr<Lane> &x) { return x->busy; });
    if (stop && pending.empty() && !busy) break;
    if (!progressed) {
      if (busy)  // poll the events again soon
        cv_work.wait_for(g, std::chrono::microseconds(50));
      else
        cv_work.wait_for(g, std::chrono::milliseconds(5), [&] { return stop || !pending.empty(); });
    }
  }
}

extern "C" {

int adanns_server_create(const adanns_index *const *indices, int nindex, int nstreams,
                         int64_t max_batch, int64_t mem_budget, adanns_server **out) {
  if (!out) return fail(ADANNS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!indices || nindex < 1 || nstreams < 1 || nstreams > 16 || max_batch < 1 ||
      max_batch > INT32_MAX || mem_budget < 0)
    return fail(ADANNS_ERR_ARG, "bad server arguments");
  for (int i = 0; i < nindex; ++i)
    if (!indices[i]) return fail(ADANNS_ERR_ARG, "index " + std::to_string(i) + " is NULL");
  auto *s = new adanns_server();
  s->indices.assign(indices, indices + nindex);
  s->max_batch = max_batch;
  s->mem_budget = mem_budget;
  cudaError_t e = cudaGetDevice(&s->device);
  for (int i = 0; i < nstreams && e == cudaSuccess; ++i) {
    auto L = std::make_unique<Lane>();
    e = cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
    s->lanes.push_back(std::move(L));
  }
  if (e != cudaSuccess) {
    for (auto &L : s->lanes) {
      if (L->done) cudaEventDestroy(L->done);
      if (L->st) cudaStreamDestroy(L->st);
    }
    delete s;
    return cuda_fail(e, "server streams");
  }
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return ADANNS_OK;
}

int adanns_server_submit(adanns_server *s, int index_slot, const float *queries, int64_t n,
                         const adanns_budget *budget, int64_t *ticket) {
  if (!s || !budget || !ticket || (n > 0 && !queries)) return fail(ADANNS_ERR_ARG, "NULL argument");
  if (index_slot < 0 || index_slot >= (int)s->indices.size())
    return fail(ADANNS_ERR_ARG, "index slot out of range");
  if (n < 1 || n > s->max_batch) return fail(ADANNS_ERR_ARG, "need 1 <= rows <= max_batch");
  const adanns_index *idx = s->indices[(size_t)index_slot];
  const adanns_budget &b = *budget;
  // the search's own argument rules, checked now so that errors surface at submit
  if (b.method != ADANNS_METHOD_IVF && b.method != ADANNS_METHOD_IVFOPQ)
    return fail(ADANNS_ERR_ARG, "unknown search method");
  if (b.k < 1 || b.k > 1024 || b.nprobe < 1 || b.nprobe > idx->nlist)
    return fail(ADANNS_ERR_ARG, "need 1 <= k <= 1024 and 1 <= nprobe <= nlist");
  if (gran_index(b.d_c) < 0 || b.d_c > idx->d_c)
    return fail(ADANNS_ERR_DIM, "d_c must be an MR granularity <= the index's clustering prefix");
  if (b.method == ADANNS_METHOD_IVF) {
    if (gran_index(b.d_s) < 0 || b.d_s > idx->d) return fail(ADANNS_ERR_DIM, "bad d_s");
    if (b.storage == ADANNS_STORE_F32 ? b.rerank_k != 0
                                      : (b.rerank_k < b.k || b.rerank_k > 2048 || b.nprobe > 128))
      return fail(ADANNS_ERR_ARG, "rerank_k / nprobe out of range for the storage tier");
  } else if (!idx->codes) {
    return fail(ADANNS_ERR_STATE, "the index has no OPQ data");
  }
  auto r = std::make_shared<Request>();
  r->slot = index_slot;
  r->b = b;
  r->n = n;
  r->q.assign(queries, queries + n * idx->d);
  r->t_arrive = now_ms();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return fail(ADANNS_ERR_STATE, "the server is shutting down");
    r->ticket = s->next_ticket++;
    if (s->t_first == 0.0) s->t_first = r->t_arrive;
    s->pending.push_back(r);
    s->live[r->ticket] = r;
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return ADANNS_OK;
}

int adanns_server_poll(adanns_server *s, int64_t ticket, int wait_ms, int64_t *ids, float *dist,
                       double *latency_ms) {
  if (!s) return fail(ADANNS_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) return fail(ADANNS_ERR_ARG, "unknown or already collected ticket");
  std::shared_ptr<Request> r = it->second;
  if (r->status == ADANNS_PENDING && wait_ms != 0) {
    auto ready = [&] { return r->status != ADANNS_PENDING; };
    if (wait_ms < 0)
      s->cv_done.wait(g, ready);
    else
      s->cv_done.wait_for(g, std::chrono::milliseconds(wait_ms), ready);
  }
  if (r->status == ADANNS_PENDING) return ADANNS_PENDING;
  s->live.erase(ticket);
  if (r->status != ADANNS_OK) return fail(r->status, r->msg);
  if (ids) memcpy(ids, r->ids.data(), sizeof(int64_t) * r->ids.size());
  if (dist) memcpy(dist, r->dist.data(), sizeof(float) * r->dist.size());
  if (latency_ms) *latency_ms = r->t_done - r->t_arrive;
  return ADANNS_OK;
}

int adanns_server_stats(adanns_server *s, double *p50_ms, double *p99_ms, int64_t *requests,
                        int64_t *batches, int64_t *queries, double *qps, int64_t *max_inflight) {
  if (!s) return fail(ADANNS_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  std::vector<double> l = s->lat_ms;
  auto pct = [&](double p) -> double {
    if (l.empty()) return 0.0;
    std::sort(l.begin(), l.end());
    // linear interpolation between closest ranks
    const double x = p / 100.0 * (double)(l.size() - 1);
    const size_t i = (size_t)x;
    const double f = x - (double)i;
    return i + 1 < l.size() ? l[i] * (1.0 - f) + l[i + 1] * f : l[i];
  };
  if (p50_ms) *p50_ms = pct(50.0);
  if (p99_ms) *p99_ms = pct(99.0);
  if (requests) *requests = s->batch_requests;
  if (batches) *batches = s->batches;
  if (queries) *queries = s->queries;
  if (qps) *qps = s->t_last > s->t_first ? 1000.0 * (double)s->queries / (s->t_last - s->t_first) : 0.0;
  if (max_inflight) *max_inflight = s->max_inflight;
  return ADANNS_OK;
}

int adanns_server_destroy(adanns_server *s) {
  if (!s) return ADANNS_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();  // drains pending and in-flight batches
  for (auto &L : s->lanes) {
    cudaEventDestroy(L->done);
    cudaStreamDestroy(L->st);
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->cv_done.notify_all();
  }
  delete s;
  return ADANNS_OK;
}

}  // extern "C"
