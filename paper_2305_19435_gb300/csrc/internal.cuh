// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/adanns.h"

struct adanns_index;

namespace adn {

constexpr uint64_t KEY_MAX = ~0ull;  // empty slot / padding key

// A probe key (coarse distance bits << 32 | list) of a masked slot: a query
// with its own, smaller nprobe than the batch's keeps its first nprobe slots
// and the rest hold PROBE_NONE, which every consumer reads as an empty list.
constexpr uint64_t PROBE_NONE = ~0ull;
__host__ __device__ inline int probe_list(uint64_t key) {
  return key == PROBE_NONE ? -1 : (int)(uint32_t)(key & 0xffffffffu);
}

// Per-query budgets of one batch (Sec. 5, compute-aware elastic search):
// device arrays of one entry per query, or null where the batch shares the
// call's value.  ds: scan prefix d_s; gi: its granularity index; np: nprobe;
// k: neighbours kept (a prefix of the batch's k results).
struct QueryBudgets {
  const int32_t *ds = nullptr, *gi = nullptr, *np = nullptr, *k = nullptr;
  QueryBudgets at(int64_t b0) const {
    QueryBudgets r;
    r.ds = ds ? ds + b0 : nullptr;
    r.gi = gi ? gi + b0 : nullptr;
    r.np = np ? np + b0 : nullptr;
    r.k = k ? k + b0 : nullptr;
    return r;
  }
};
// slots at or past np[q] of each query's nprobe probe keys -> PROBE_NONE
int launch_mask_probes(uint64_t *ckeys, int64_t B, int nprobe, const int32_t *np, cudaStream_t st);
// entries at or past k[q] of each row of k_max results -> (-1, +inf)
int launch_pad_rows(int64_t *ids, float *dist, int64_t B, int k_max, const int32_t *k,
                    cudaStream_t st);

// bits of an index's sticky device error word (adanns_index_status); the low
// byte is the tensor-core pipeline stage whose wait timed out
constexpr int ADANNS_DEVERR_RERANK = 0x100;  // rerank pair outside its member chunk

// A candidate is packed as (float bits of a non-negative distance) << 32 | id,
// so unsigned order is (distance, id) order.
__host__ __device__ inline uint64_t pack_key(float d, uint32_t id) {
#ifdef __CUDA_ARCH__
  return ((uint64_t)__float_as_uint(d) << 32) | id;
#else
  union { float f; uint32_t u; } c;
  c.f = d;
  return ((uint64_t)c.u << 32) | id;
#endif
}

// MR granularities (Sec. 3: nested sizes 8 .. 2048)
constexpr int NGRAN = 14;
extern const int kGran[NGRAN];
int gran_index(int m);  // index in kGran, or -1

inline int pad16(int x) { return (x + 15) & ~15; }

// kGran[g] on the device
__device__ __forceinline__ int kGranDev(int g) {
  switch (g) {
    case 0: return 8;
    case 1: return 16;
    case 2: return 32;
    case 3: return 48;
    case 4: return 64;
    case 5: return 96;
    case 6: return 128;
    case 7: return 192;
    case 8: return 256;
    case 9: return 384;
    case 10: return 512;
    case 11: return 768;
    case 12: return 1024;
    default: return 2048;
  }
}


// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
#define ADN_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return ::adn::cuda_fail(e__, #call); \
  } while (0)
extern std::atomic<long long> g_launches;  // kernels launched since load
#define ADN_LAUNCH(what)                                 \
  do {                                                   \
    ::adn::g_launches.fetch_add(1, std::memory_order_relaxed); \
    cudaError_t e__ = cudaGetLastError();                \
    if (e__ != cudaSuccess) return ::adn::cuda_fail(e__, what); \
  } while (0)

// ---------------------------------------------------------------- scratch
// The library's own stream-ordered memory pool for the current device: its
// release threshold is unlimited, so scratch freed at the end of one call is
// reused by the next without returning memory to the driver.
cudaMemPool_t scratch_pool();
// Bytes of scratch one search call may hold at once (ADANNS_OPT_SCRATCH_BYTES).
int64_t scratch_budget();
// Runtime options (ADANNS_OPT_*): current value; take_option returns it and
// stores `reset` (one-shot test hooks); set_option validates.
int64_t option(int opt);
int64_t take_option(int opt, int64_t reset);
int set_option(int opt, int64_t value);
int64_t max_probe_members(const adanns_index *idx, int nprobe);

// Stream-ordered scratch allocation from that pool on the call's stream.
struct Scratch {
  cudaStream_t st;
  void *ptrs[64];
  int n = 0;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], st);
  }
  template <class T>
  int get(T **out, size_t count) {
    void *p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = scratch_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st)
                         : cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess || n >= 64) {
      cudaGetLastError();
      if (p) cudaFreeAsync(p, st);
      return fail(ADANNS_ERR_OOM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
    }
    ptrs[n++] = p;
    *out = (T *)p;
    return ADANNS_OK;
  }
};

// ---------------------------------------------------------------- scan
// One distance-plus-top-k pass over (list, query-tile) work items.
// Vectors are stored prefix-major: list l's block b (dims [16b, 16b+16)) is a
// contiguous [n_l][16] slab at float offset list_off[l]*d_pad + b*16*n_l.
struct ScanArgs {
  const float *xpm;        // prefix-major storage
  int d_pad;               // stored floats per vector (multiple of 16)
  int dims;                // dimensions used (multiple of 4, <= d_pad)
  const int64_t *list_off; // member offset of each list (nlist + 1)
  const int32_t *list_ids; // id of each member (NULL: the member index)
  const float *mscale;     // per-member scale in list order (NULL: 1)
  const float *qn;         // prepared queries, rows of ldq floats (16-byte aligned)
  int ldq;
  // work items: either explicit tiles or a dense sweep of nq queries over list 0
  const int32_t *tile_list, *tile_beg, *tile_cnt;
  const int *ntiles_dev;   // device count of explicit tiles
  int nq;                  // dense mode: number of queries
  int *counter;            // zeroed work counter
  const int32_t *pair_q;   // query row of each pair (NULL: pair index)
  const int32_t *pair_out; // output row of each pair (NULL: pair index)
  int k;
  uint64_t *out_keys;      // [row][k] sorted keys (KEY_MAX padding)
  int grid;                // CTAs to launch
  int tq;                  // queries per thread (QT = 16 tq); 0 = by k
  int nsplit;              // explicit tiles: member ranges per tile (0 or 1: whole list);
                           // item t = (tile t / nsplit, range t % nsplit), output row
                           // pair_out * nsplit + range
};
int launch_scan_f32(const ScanArgs &a, cudaStream_t st);
int scan_query_tile(int k, int tq = 0);  // queries per work item

// Autotuned choices for a shape bucket (device, k, d_s, queries per probed
// list): queries per thread of the tiled FP32 list scan (4 or 1), TUNE_STREAM
// for the streaming scan, 0 when not tuned.
constexpr int TUNE_STREAM = 16;
int tuned_scan_tq(int k, int d_s, double queries_per_list);
// Autotuned tile of the BF16 / FP8 tensor-core list scan for a bucket (device,
// tier, d_s, queries per probed list): 128 (128 queries x 256 members) or
// MMA_NARROW_QT (128 members x 32 queries); 0 when not tuned.  which: 0 BF16,
// 1 FP8.
int tuned_lowp_qt(int which, int d_s, double queries_per_list);

// ---------------------------------------------------------------- helpers
// dims_b_q (or null): a per-query dims_b for the second copy; rows (or null):
// prepared row i is query row rows[i] of q
int launch_prep_queries(const float *q, int64_t B, int ld, int dims_a, int dims_b, int metric,
                        float *qa, int lda, float *qb, int ldb, cudaStream_t st,
                        const int32_t *dims_b_q = nullptr, const int32_t *rows = nullptr);
int launch_keys_to_result(const uint64_t *keys, int64_t rows, int k, int64_t *ids, int32_t *ids32,
                          float *dist, cudaStream_t st);
int launch_invert_probes(const uint64_t *ckeys, int64_t B, int nprobe, int nlist, int qt,
                         int32_t *lcnt, int32_t *lbeg, int32_t *lfill, int32_t *tbeg,
                         int32_t *pair_q, int32_t *pair_out, int32_t *tile_list,
                         int32_t *tile_beg, int32_t *tile_cnt, int *ntiles, int32_t *probes_out,
                         cudaStream_t st);
// The same over probe slots [s0, s0 + ns) of each query only (pair_out still
// holds the pair index q * nprobe + slot; probes_out gets those slots' lists).
int launch_invert_probe_slots(const uint64_t *ckeys, int64_t B, int nprobe, int s0, int ns,
                              int nlist, int qt, int32_t *lcnt, int32_t *lbeg, int32_t *lfill,
                              int32_t *tbeg, int32_t *pair_q, int32_t *pair_out,
                              int32_t *tile_list, int32_t *tile_beg, int32_t *tile_cnt,
                              int *ntiles, int32_t *probes_out, cudaStream_t st);
// Per-query budgets in the merge (all null: none): ckeys / nsplit mark the runs
// of masked probe slots, kq the per-query k, orow each query's output row.
struct MergeMask {
  const uint64_t *ckeys = nullptr;
  int nsplit = 1;
  const int32_t *kq = nullptr, *orow = nullptr;
};
int launch_merge(const uint64_t *pkeys, int64_t B, int nprobe, int k, int64_t *out_ids,
                 float *out_dist, cudaStream_t st, const MergeMask &mm = MergeMask{});
int num_sms();
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (device, kernel, size)
cudaError_t ensure_smem(const void *fn, size_t bytes);

// ---------------------------------------------------------------- build
int launch_gather_normalize(const float *x, int64_t n, int ld, const int64_t *rows, int dim,
                            int metric, float *out, int ldo, cudaStream_t st);
int launch_prefix_major(const float *x, int ld, int d, int d_pad, const int64_t *list_off,
                        const int32_t *list_ids, const int32_t *assign, int64_t N, float *xpm,
                        cudaStream_t st);
int launch_inv_norms(const float *x, int ld, int d, const int32_t *list_ids, int64_t N,
                     int metric, float *invn /* [ng][N] */, int ng, cudaStream_t st);
int launch_kmeans_update(const float *t, int64_t n, int ld, int dim, const int32_t *assign,
                         int nc, double *sums, int32_t *counts, float *cent, cudaStream_t st);
int launch_sum_keys(const uint64_t *keys, int64_t n, double *out, cudaStream_t st);
int launch_positions(const int32_t *list_ids, int64_t N, int32_t *pos, cudaStream_t st);
int check_assignment(const int32_t *a, int64_t n, int nlist, cudaStream_t st);
int build_csr(const int32_t *assign, int64_t N, int nlist, int64_t *list_off, int32_t *list_ids,
              cudaStream_t st);

// ---------------------------------------------------------------- profiling
enum Stage {
  ST_PREP = 0, ST_COARSE = 1, ST_INVERT = 2, ST_SCAN = 3, ST_MERGE = 4, ST_LUT = 5, ST_ADC = 6,
  ST_RERANK = 7, ST_MMA = 8, ST_SELECT = 9, ST_RR_SORT = 10, ST_RR_PAIRS = 11, ST_RR_FINAL = 12,
  ST_NSTAGE = 16
};

// Tensor-core list scan of the mixed-precision path (mma_scan.cu).
// queries per tile of the narrow tensor-core scan (tiles of 128 members x this)
constexpr int MMA_NARROW_QT = 32;
struct MmaScanArgs {
  const int32_t *tile_list, *tile_beg, *tile_cnt;
  const int *ntiles_dev;
  const int64_t *list_off;
  const int32_t *pair_out;   // pair index (q * nprobe + slot) of each tile row
  const int64_t *pbase;      // candidate segment start of each pair (multiple of 8)
  int64_t pstride;           // > 0: key segment of pair p at (p / nprobe) * pstride instead
                             // (one segment per query: a scan of the nearest list only)
  const float *cx;           // per member (list order): s_x * nu_x(d_s), 0 for a zero prefix
  const float *qn2;          // per query: |P_ds(q)|^2
  const float *qsc;          // per query: operand scale s_q
  int nprobe;
  int nkb;                   // K-blocks of the d_s prefix
  int d_blocks;              // storage blocks per vector
  uint16_t *cand;            // 16-bit fixed-point approximate distance keys
  const float *x2;           // per member: squared norm of the used prefix (NULL: 1, or 0 for
                             // a zero prefix, as for normalised prefixes)
  int *err;
  int *tile_counter;         // zeroed before the launch: next tile to take
  int fp8;
  int few;                   // few queries per probed list (memory-bound): FP8 takes the
                             // four-stage ring with narrow key staging, as BF16 does
  // filtered mode (rec != NULL, tau != NULL): instead of every key, each
  // (query, probe slot) pair p keeps only its members with key <= tau[query],
  // as 32-bit records (key << 16 | member index, lists below 65,537 members)
  // compacted from rec[pbase[p]]; the CTA counts them per tile row in shared
  // memory and writes the count to rcnt[p] once the pair's work item is done
  // (rcnt zeroed before, for pairs of empty lists)
  uint32_t *rec;
  int *rcnt;
  const uint16_t *tau;
  uint64_t wait_ns;          // bound of each pipeline wait (set by the launcher)
  int skip_fill;             // test hook: stage load skip_fill of work item 0 is left out (-1: none)
};
// work counters recorded while profiling is on (adanns_profile_read_counters)
enum ProfileCounter {
  PC_RERANK_PAIRS = 0, PC_SHORTLIST_SLOTS = 1, PC_SURVIVORS = 2, PC_SELECT_SLOW = 3,
  PC_NCOUNTER = 8
};
bool profiling();  // whether adanns_profile_enable(1) is in effect
void profile_count(int counter, const int64_t *dev_value, cudaStream_t st);
void profile_count_host(int counter, int64_t value);

// Cluster mapping for d_c <= 64 and n_p <= 64: out[q][0:k] = the k smallest
// (distance, list) keys of the query rows qc [B][ldq] against the row-major
// centroids (first d_c of ldc columns).  Returns 1, launching nothing, for
// other shapes (the caller then uses the general scan kernel).
int launch_coarse(const float *cent, int ldc, int nlist, int d_c, const float *qc, int ldq,
                  int64_t B, int k, uint64_t *out, cudaStream_t st);
// Cluster mapping on the tensor cores with the same result: BF16 products of
// the query and centroid prefixes shortlist every centroid that can be among
// the k nearest (a bound on the quantisation error), which are then scored
// exactly in FP32 as above.  Returns 1, launching nothing, when the index has
// no BF16 centroid copy, has fewer than 256 lists, d_c > 64, k > 1024, or
// k > 32 with more than 16,384 lists.
int launch_coarse_tc(const adanns_index *idx, const float *qc, int ldq, int64_t B, int d_c, int k,
                     uint64_t *out, cudaStream_t st);
// Both, in order of preference, then the general scan over the prefix-major
// centroid table (counter: the scan's work counter, zeroed by the caller).
int run_coarse(const adanns_index *idx, const float *qc, int ldq, int64_t B, int d_c, int k,
               uint64_t *out, int *counter, cudaStream_t st);
constexpr int64_t CT_SLICE_MIN = 4096;  // fewest points per tensor-core assignment slice
int build_centroid_lowp(adanns_index *x, cudaStream_t st);
// Candidate segments of a batch: per query, the probed lists' sizes rounded
// up to 8, laid end to end (qtot: per-query total, qbase: its start, pbase:
// start of each (query, probe) segment).
int launch_cand_segments(const uint64_t *ckeys, int64_t B, int nprobe, const int64_t *list_off,
                         int64_t *qtot, int64_t *qbase, int64_t *pbase, cudaStream_t st);
// Per query, the kk smallest 32-bit keys (order-preserving: non-negative
// FP32 distance bits) of its candidate segments, written as
// (key << 32 | database id), KEY_MAX padding; ties at the cut go to the
// smallest candidate positions.  nprobe <= 256.
int launch_scan_i32(const int32_t *v, int64_t n, int32_t *out, cudaStream_t st);
int launch_scan64(const int64_t *in, int64_t n, int64_t *out, int64_t *total, cudaStream_t st);
// the streaming FP32 scan for this batch shape (the autotuned choice when the
// bucket is tuned, else few queries per probed list)
bool fp32_stream_enabled(double queries_per_list, int nprobe, int k = 0, int d_s = 0);
// scratch bytes of search_f32_stream for these arguments (host arithmetic)
int64_t stream_scratch_bytes(const adanns_index *idx, int64_t B, int d_c, int d_s, int nprobe,
                             int k);
// The tiled FP32 scan (many queries per probed list).  qb (or null): per-query
// nprobe / k at most the call's, one d_s for the batch; rows (or null): query
// i of the batch is row rows[i] of `queries` and its results go to output row
// rows[i] (rows of k entries).
int search_f32_tiled(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                     int nprobe, int k, int64_t *out_ids, float *out_dist, int32_t *out_probes,
                     cudaStream_t st, const QueryBudgets *qb = nullptr,
                     const int32_t *rows = nullptr);
// qb (or null): per-query d_s / nprobe / k at most the call's d_s, nprobe, k
int search_f32_stream(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                      int nprobe, int k, int64_t *out_ids, float *out_dist, int32_t *out_probes,
                      cudaStream_t st, const QueryBudgets *qb = nullptr);
int launch_select16(const uint16_t *cand, const uint64_t *ckeys, int nprobe, const int64_t *qbase,
                    const int64_t *list_off, int kk, int k, const float *qrho, float rmax,
                    float e_rest, int prune, int64_t B, int64_t *out, unsigned long long *stats,
                    cudaStream_t st);
// Filtered tensor-core scan: from the keys of each query's nearest list
// (cand0 + q * stride0, the list of probe slot 0), tau = their kk-th smallest
// (0xFFFF with fewer than kk members) and slot 0's records with key <= tau;
// then the shortlist selected from the survivors (same result as
// launch_select16).
int launch_shortlist_tau(const uint16_t *cand0, int64_t stride0, const uint64_t *ckeys,
                         const int64_t *list_off, uint32_t *rec, int *rcnt, const int64_t *pbase,
                         int nprobe, int kk, int64_t B, uint16_t *tau, cudaStream_t st);
// stats (NULL, or 2 zeroed device counters): survivors, queries selected
// from global memory because their survivors exceed the shared buffer
int launch_select_surv(const uint32_t *rec, const int *rcnt, const int64_t *pbase,
                       const uint64_t *ckeys, int nprobe, const int64_t *list_off, int kk, int k,
                       const float *qrho, float rmax, float e_rest, int prune, int64_t B,
                       int64_t *out, unsigned long long *stats, cudaStream_t st);
int launch_keys_to_ids(const uint64_t *keys, int64_t n, int64_t *ids, cudaStream_t st);
int launch_final_topk(const uint64_t *keys, int kr, int64_t B, int k, int64_t *out_ids,
                      float *out_dist, cudaStream_t st);
int adc_dist_query_tile(int M);
// res_S / res_w / res_w2 / z (NULL for plain codes): residual terms and the
// queries' rotated vectors [B][d_s]; the score of a member of list l is then
// sum_m (lut_q[m][c_m] + S_l[m][c_m]) + w2_l - 2 <w_l, z_q>
int launch_adc_dist(const uint8_t *codes, const int64_t *list_off, int M, const float *lut,
                    const int32_t *tl, const int32_t *tb, const int32_t *tc, const int *ntiles,
                    int *counter, const int32_t *pair_q, const int32_t *pair_out,
                    const int64_t *pbase, uint32_t *cand, int qa, int nsplit, cudaStream_t st,
                    const float *res_S = nullptr, const float *res_w = nullptr,
                    const float *res_w2 = nullptr, const float *z = nullptr, int d_s = 0);
int launch_select32(const uint32_t *cand, const uint64_t *ckeys, int nprobe, const int64_t *qbase,
                    const int64_t *list_off, const int32_t *list_ids, int64_t B, int kk,
                    uint64_t *out, cudaStream_t st);

// Records an event pair around its scope on `st` when profiling is enabled.
class StageTimer {
 public:
  StageTimer(int stage, cudaStream_t st);
  ~StageTimer();

 private:
  int stage_;
  cudaStream_t st_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  double t0_ = 0.0;
};

int build_lowp(adanns_index *x, const float *db, int which, cudaStream_t st);
// chunk-table slot of a rerank member-chunk size (64, 32, 16, 8)
inline int rerank_chunk_index(int mc) { return mc >= 64 ? 0 : mc >= 32 ? 1 : mc >= 16 ? 2 : 3; }
// the rerank work order and chunk tables of an index (host copies of the
// centroids and list offsets; synchronises the stream)
int build_rerank_order(adanns_index *x, cudaStream_t st);
// qb (or null): per-query nprobe / k at most the call's (d_s is the batch's)
int search_mixed(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                 int nprobe, int k, int which, int kk, int64_t *out_ids, float *out_dist,
                 int32_t *out_probes, cudaStream_t st, const QueryBudgets *qb = nullptr);

}  // namespace adn

// Index (opaque in the C ABI)
struct adanns_index {
  int64_t N = 0;
  int d = 0, d_pad = 0, d_c = 0, dc_pad = 0, nlist = 0, metric = 0, storage = 0;
  int max_list = 0;
  float *centroids = nullptr;   // nlist x d_c row-major
  // BF16 copy of the centroids for the tensor-core cluster mapping (metric
  // L2_PREFIXNORM): blocks of 64 coordinates [block][centroid][64], the
  // per-centroid scale, squared prefix norms [granularity][nlist], and per
  // granularity the largest absolute quantisation residual |(c - s c~)[0:g]|
  // and the largest centroid norm (host copies)
  void *cent_low = nullptr;
  int cent_low_blocks = 0;
  float *cent_sc = nullptr;
  float *cent_n2 = nullptr;
  float cent_rmax[adn::NGRAN] = {};
  float cent_maxnorm = 0.f;
  float *cent_pm = nullptr;     // centroids prefix-major, one list of nlist members
  int64_t *cent_off = nullptr;  // {0, nlist}
  int64_t *list_off = nullptr;  // nlist + 1
  int32_t *list_ids = nullptr;  // N
  float *xpm = nullptr;         // prefix-major FP32 vectors
  float *invn = nullptr;        // [ng][N] inverse prefix norms in list order
  int ng = 0;
  int32_t *assign = nullptr;    // list of each id (N)
  int32_t *pos_of_id = nullptr; // list-order position of each id (N)
  // OPQ on the d_s prefix (adanns_build_opq / adanns_index_set_opq)
  int opq_ds = 0, opq_M = 0;
  float *opq_R = nullptr;       // d_s x d_s, z = x R
  float *opq_C = nullptr;       // M x 256 x (d_s / M)
  uint8_t *codes = nullptr;     // N x M, list order
  // residual codes (adanns_build_opq_residual / adanns_index_set_opq_residual):
  // lcent = list centres [nlist][d_s] (mean normalised d_s prefix of each
  // list), w = lcent R [nlist][d_s], w2 = |w_l|^2 [nlist], S[l][m][c] =
  // 2 <w_l,m, C_m[c]> [nlist][M][256]; NULL for plain codes
  float *opq_lcent = nullptr, *opq_w = nullptr, *opq_w2 = nullptr, *opq_S = nullptr;
  // low-precision tiers [0] BF16 (64-dim blocks), [1] FP8-E4M3 (128-dim blocks)
  void *lowp[2] = {nullptr, nullptr};
  int lowp_blocks[2] = {0, 0};
  float *lowp_sx[2] = {nullptr, nullptr};  // per-vector scale, list order
  float *lowp_cx[2] = {nullptr, nullptr};  // [ng][N] scale * inverse prefix norm
  // per granularity g: max over members of nu_g(x) * |(x - s_x x~)[0:g]|, the
  // largest relative quantisation residual of a normalised prefix (host copy)
  float lowp_rmax[2][adn::NGRAN] = {};
  // rerank work order: lists in a nearest-neighbour chain of the centroids,
  // cut into member chunks of 64 / 32 / 16 / 8; rr_cmap[ci][c] = (list, first
  // member, list offset, list size) of chunk c in that order, so that a
  // rerank CTA finds its chunk and list with one load, and rr_chunks[ci] the
  // chunk count
  int4 *rr_cmap[4] = {nullptr, nullptr, nullptr, nullptr};
  int rr_chunks[4] = {0, 0, 0, 0};
  int64_t *h_list_off = nullptr;  // host copy of list offsets
  int *dev_err = nullptr;         // sticky device status word (tensor-core pipeline timeouts)
};
