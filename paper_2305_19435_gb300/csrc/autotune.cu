// Autotuners for the exact FP32 list scan and for the tile shape of the
// BF16 / FP8 tensor-core list scan.
//
// The tunable is the scan kernel and its work-item shape: the tiled scan with
// 64 queries per (list, query-tile) item and a 4 x 8 register tile per
// thread, the tiled scan with 16 queries and a 1 x 8 tile, or the streaming
// scan (each member row read once per group of 4 queries, distances selected
// afterwards).  The first amortises each list block over more queries
// (batched regime); the second needs a quarter of the top-k buffers, so more
// CTAs stay resident when few queries share a list; the third suits lists
// probed by a handful of queries (serving).  Their crossover depends on d_s,
// k and the batch, so adanns_autotune_search times all three on the caller's
// real batch with CUDA events and records the fastest under a bucket key
// (device, k rounded up to a power of two, d_s, log2 of queries per probed
// list); adanns_search_ivf then uses the recorded choice for matching calls.
// All three give the same results.
//
// The BF16 / FP8 tensor-core list scan has two tile shapes: 128 queries x 256
// members (each member tile feeds a whole query tile: the batched regime) and
// 128 members x 32 queries (a tile's stage is nearly all database bytes when a
// list is probed by a handful of queries).  adanns_autotune_search_lowp times
// both on the caller's batch and records the faster under (device, tier, d_s,
// log2 of queries per probed list); the low-precision search uses it in place
// of its built-in rule.
#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "internal.cuh"

namespace adn {

namespace {
std::mutex g_tmu;
std::map<std::string, int> g_table;
thread_local int g_force_tq = 0;
thread_local int g_force_qt = 0;

std::string device_tag() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string name = p.name;
  for (auto &ch : name)
    if (ch == ' ') ch = '_';
  return name + "-" + std::to_string(p.multiProcessorCount);
}

std::string bucket_key(int k, int d_s, double qpl) {
  int kp = 1;
  while (kp < k) kp <<= 1;
  const int qb = (int)std::floor(std::log2(qpl + 1.0));
  return device_tag() + "|k" + std::to_string(kp) + "|ds" + std::to_string(d_s) + "|q" +
         std::to_string(qb);
}
std::string lowp_key(int which, int d_s, double qpl) {
  const int qb = (int)std::floor(std::log2(qpl + 1.0));
  return device_tag() + "|lp" + (which == 1 ? "fp8" : "bf16") + "|ds" + std::to_string(d_s) +
         "|q" + std::to_string(qb);
}

bool valid_entry(const std::string &key, int v) {
  if (key.find("|lp") != std::string::npos) return v == 128 || v == MMA_NARROW_QT;
  return v == 1 || v == 4 || v == TUNE_STREAM;
}
}  // namespace

int tuned_lowp_qt(int which, int d_s, double queries_per_list) {
  if (g_force_qt) return g_force_qt;
  std::lock_guard<std::mutex> g(g_tmu);
  if (g_table.empty()) return 0;
  auto it = g_table.find(lowp_key(which, d_s, queries_per_list));
  return it == g_table.end() ? 0 : it->second;
}

int tuned_scan_tq(int k, int d_s, double queries_per_list) {
  if (g_force_tq) return g_force_tq;
  std::lock_guard<std::mutex> g(g_tmu);
  if (g_table.empty()) return 0;
  auto it = g_table.find(bucket_key(k, d_s, queries_per_list));
  return it == g_table.end() ? 0 : it->second;
}

}  // namespace adn

using namespace adn;

extern "C" {

int adanns_autotune_search(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                           int d_s, int nprobe, int k, int64_t *out_ids, float *out_dist,
                           void *cuda_stream, int *chosen, float *best_ms) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (B < 1) return fail(ADANNS_ERR_ARG, "need a non-empty batch");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0, e1;
  ADN_CUDA(cudaEventCreate(&e0));
  ADN_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_t = 0.f;
  int rc = ADANNS_OK;
  const int cands[3] = {4, 1, TUNE_STREAM};
  for (int ci = 0; ci < 3 && rc == ADANNS_OK; ++ci) {
    const int tq = cands[ci];
    if (tq == 4 && k > 128) continue;
    if (tq == TUNE_STREAM && (nprobe > 256 || !option(ADANNS_OPT_FP32_STREAM))) continue;
    g_force_tq = tq;
    rc = adanns_search_ivf(idx, queries, B, d_c, d_s, nprobe, k, ADANNS_STORE_F32, 0, out_ids,
                           out_dist, nullptr, cuda_stream);
    if (rc) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && rc == ADANNS_OK; ++r)
      rc = adanns_search_ivf(idx, queries, B, d_c, d_s, nprobe, k, ADANNS_STORE_F32, 0, out_ids,
                             out_dist, nullptr, cuda_stream);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.f;
    if (best == 0 || ms < best_t) {
      best = tq;
      best_t = ms;
    }
  }
  g_force_tq = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> g(g_tmu);
    g_table[bucket_key(k, d_s, (double)B * nprobe / idx->nlist)] = best;
  }
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = best_t;
  return ADANNS_OK;
}

int adanns_autotune_search_lowp(const adanns_index *idx, const float *queries, int64_t B,
                                int d_c, int d_s, int nprobe, int k, int storage, int rerank_k,
                                int64_t *out_ids, float *out_dist, void *cuda_stream,
                                int *chosen, float *best_ms) {
  if (!idx) return fail(ADANNS_ERR_ARG, "index is NULL");
  if (B < 1) return fail(ADANNS_ERR_ARG, "need a non-empty batch");
  if (storage != ADANNS_STORE_BF16 && storage != ADANNS_STORE_FP8E4M3)
    return fail(ADANNS_ERR_ARG, "autotune_search_lowp: storage must be BF16 or FP8-E4M3");
  if (option(ADANNS_OPT_NARROW_SCAN) != 1)
    return fail(ADANNS_ERR_ARG,
                "autotune_search_lowp: ADANNS_OPT_NARROW_SCAN fixes the tile shape (set it to 1)");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0, e1;
  ADN_CUDA(cudaEventCreate(&e0));
  ADN_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_t = 0.f;
  int rc = ADANNS_OK;
  const int cands[2] = {128, MMA_NARROW_QT};
  for (int ci = 0; ci < 2 && rc == ADANNS_OK; ++ci) {
    g_force_qt = cands[ci];
    rc = adanns_search_ivf(idx, queries, B, d_c, d_s, nprobe, k, storage, rerank_k, out_ids,
                           out_dist, nullptr, cuda_stream);
    if (rc) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && rc == ADANNS_OK; ++r)
      rc = adanns_search_ivf(idx, queries, B, d_c, d_s, nprobe, k, storage, rerank_k, out_ids,
                             out_dist, nullptr, cuda_stream);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.f;
    if (best == 0 || ms < best_t) {
      best = cands[ci];
      best_t = ms;
    }
  }
  g_force_qt = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const int which = storage == ADANNS_STORE_FP8E4M3 ? 1 : 0;
  {
    std::lock_guard<std::mutex> g(g_tmu);
    g_table[lowp_key(which, d_s, (double)B * nprobe / idx->nlist)] = best;
  }
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = best_t;
  return ADANNS_OK;
}

int adanns_tune_save(const char *path) {
  if (!path) return fail(ADANNS_ERR_ARG, "path is NULL");
  std::lock_guard<std::mutex> g(g_tmu);
  std::ofstream f(path);
  if (!f) return fail(ADANNS_ERR_ARG, std::string("cannot write ") + path);
  for (auto &kv : g_table) f << kv.first << " " << kv.second << "\n";
  return ADANNS_OK;
}

int adanns_tune_clear(void) {
  std::lock_guard<std::mutex> g(g_tmu);
  g_table.clear();
  return ADANNS_OK;
}

int adanns_tune_load(const char *path) {
  if (!path) return fail(ADANNS_ERR_ARG, "path is NULL");
  std::ifstream f(path);
  if (!f) return fail(ADANNS_ERR_ARG, std::string("cannot read ") + path);
  std::lock_guard<std::mutex> g(g_tmu);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream ss(line);
    std::string key;
    int tq = 0;
    if (ss >> key >> tq && valid_entry(key, tq)) g_table[key] = tq;
  }
  return ADANNS_OK;
}

}  // extern "C"
