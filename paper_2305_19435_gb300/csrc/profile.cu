// Optional per-stage timing with CUDA events recorded on the launching stream.
// Off by default; when on, every profiled stage of every call records an event
// pair around its launches, and adanns_profile_read sums the elapsed times.
#include <chrono>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace adn {

namespace {
struct Rec {
  int stage;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
double g_host_us[ST_NSTAGE] = {0};

// work counters: device values copied (stream-ordered) into device slots
constexpr int NSLOT = 1 << 16;
int64_t *g_slots = nullptr;
int g_nslot = 0;
std::vector<int> g_slot_counter;
int64_t g_host_cnt[PC_NCOUNTER] = {0};

double now_us() {
  return std::chrono::duration<double, std::micro>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

bool profiling() {
  std::lock_guard<std::mutex> g(g_mu);
  return g_on;
}

void profile_count(int counter, const int64_t *dev_value, cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_on || counter < 0 || counter >= PC_NCOUNTER) return;
  if (!g_slots && cudaMalloc(&g_slots, sizeof(int64_t) * NSLOT) != cudaSuccess) {
    cudaGetLastError();
    g_slots = nullptr;
    return;
  }
  if (g_nslot >= NSLOT) return;
  if (cudaMemcpyAsync(g_slots + g_nslot, dev_value, sizeof(int64_t), cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return;
  }
  g_slot_counter.push_back(counter);
  ++g_nslot;
}

void profile_count_host(int counter, int64_t value) {
  std::lock_guard<std::mutex> g(g_mu);
  if (g_on && counter >= 0 && counter < PC_NCOUNTER) g_host_cnt[counter] += value;
}

StageTimer::StageTimer(int stage, cudaStream_t st) : stage_(stage), st_(st) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_on) return;
  t0_ = now_us();
  a_ = take_event();
  b_ = take_event();
  if (a_ && b_) cudaEventRecord(a_, st_);
}

StageTimer::~StageTimer() {
  std::lock_guard<std::mutex> g(g_mu);
  if (!a_ || !b_) return;
  if (stage_ >= 0 && stage_ < ST_NSTAGE) g_host_us[stage_] += now_us() - t0_;
  cudaEventRecord(b_, st_);
  g_recs.push_back({stage_, a_, b_});
}

}  // namespace adn

using namespace adn;

extern "C" {

int adanns_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_mu);
  for (auto &r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  for (int i = 0; i < ST_NSTAGE; ++i) g_host_us[i] = 0.0;
  for (int i = 0; i < PC_NCOUNTER; ++i) g_host_cnt[i] = 0;
  g_nslot = 0;
  g_slot_counter.clear();
  g_on = on != 0;
  return ADANNS_OK;
}

int adanns_profile_read_host(double *us, int nstage) {
  if (!us || nstage < 1) return fail(ADANNS_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(g_mu);
  for (int i = 0; i < nstage; ++i) us[i] = i < ST_NSTAGE ? g_host_us[i] : 0.0;
  return ADANNS_OK;
}

int adanns_profile_read(double *ms, int64_t *count, int nstage) {
  if (!ms || !count || nstage < 1) return fail(ADANNS_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(g_mu);
  for (int i = 0; i < nstage; ++i) {
    ms[i] = 0.0;
    count[i] = 0;
  }
  for (auto &r : g_recs) {
    if (r.stage < 0 || r.stage >= nstage) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "profile event");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "profile elapsed");
    ms[r.stage] += t;
    count[r.stage] += 1;
  }
  return ADANNS_OK;
}

int adanns_profile_read_counters(int64_t *values, int ncounter) {
  if (!values || ncounter < 1) return fail(ADANNS_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(g_mu);
  for (int i = 0; i < ncounter; ++i) values[i] = i < PC_NCOUNTER ? g_host_cnt[i] : 0;
  if (g_nslot > 0) {
    std::vector<int64_t> h(g_nslot);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
      e = cudaMemcpy(h.data(), g_slots, sizeof(int64_t) * g_nslot, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "profile counters");
    for (int i = 0; i < g_nslot; ++i)
      if (g_slot_counter[i] < ncounter) values[g_slot_counter[i]] += h[i];
  }
  return ADANNS_OK;
}

}  // extern "C"
