// Exact FP32 distance scan with a fused streaming top-k.
//
// One kernel serves three steps of AdANNS-IVF (Algorithm 1):
//   * cluster mapping: every query against the centroid table at d_c, keep
//     the n_p nearest (computeDistances + sortAscending[:num_probes]);
//   * the Lloyd assignment of the k-means builder (k = 1);
//   * the linear scan of the probed lists at d_s, keep the k nearest
//     (linearScan(q, candidates, d_search, k)).
//
// Work item = (list, up to QT queries that probe it).  The CTA streams the
// list's members in chunks of XT through shared memory, one 16-dim prefix
// block at a time (the prefix-major layout makes each block of a chunk one
// contiguous 8 KB read), and forms the QT x XT tile of
//     dist = sum_j (q_j - s_x * x_j)^2
// in registers (difference form: no cancellation for near neighbours).
// Distances never leave the SM: each query keeps a shared-memory candidate
// buffer; a candidate enters only if its key beats the query's current k-th
// key, and a warp sorts and trims the buffer when it fills.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {

namespace {
constexpr int THREADS = 256;
constexpr int XT = 128;      // members per chunk
constexpr int XROW = 20;     // padded floats per 16-float smem row (conflict-free float4 reads)
// cp.async pipeline depth over prefix blocks: 2 for the 64-query tile (the
// batched regime, compute-bound), 4 for the 16-query tile (few queries per
// list: memory-bound, so more blocks in flight)
constexpr int nstage_for(int tq) { return tq == 1 ? 4 : 2; }
constexpr int ROUND = 32;    // candidates appended per query between compactions
constexpr int NWARP = THREADS / 32;

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct ScanCfg {
  int tq;    // queries per thread (QT = 16 * tq)
  int cap;   // candidate buffer per query (0: top-1 mode)
  size_t smem;
};

// shared memory: [X stages | merge scratch] [Q stages] ids scales qrow orow cnt nsorted tau buf
size_t smem_bytes(int qt, int cap) {
  const int NSTAGE = nstage_for(qt / 16);
  size_t xs = (size_t)NSTAGE * XT * XROW * 4;
  size_t scratch = (size_t)NWARP * cap * 8;
  size_t s = xs > scratch ? xs : scratch;
  s += (size_t)NSTAGE * qt * XROW * 4;
  s += XT * 4 * 2;
  s += qt * 4 * 4;
  s = (s + 7) & ~(size_t)7;
  s += qt * 8;
  s += (size_t)qt * cap * 8;
  return s;
}

ScanCfg choose(int k, int tq) {
  ScanCfg c;
  if (k == 1) {
    c.tq = 4;
    c.cap = 0;
    c.smem = smem_bytes(64, 0);
    return c;
  }
  const int kp = next_pow2(k);
  // buffer slack: a query compacts only when its next round could overflow;
  // small k (the cluster mapping) can afford room for several rounds, so the
  // sort-and-merge runs a few times per work item instead of every round
  const int slack = kp <= 32 ? 4 : (kp <= 64 ? 2 : 1);
  c.cap = kp + ROUND * slack;
  c.tq = kp <= 128 ? 4 : 1;
  if (tq == 1) c.tq = 1;  // a smaller query tile is valid for every k
  c.smem = smem_bytes(16 * c.tq, c.cap);
  return c;
}

// number of keys in sorted a[0:n) that are < key
__device__ __forceinline__ int lower_bound_u64(const uint64_t *a, int n, uint64_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// buf[0:na) is sorted, buf[na:n) is not: sort the new keys, merge the two runs
// (each key's output rank = its own index + the count of smaller keys in the
// other run; keys are unique), keep the k smallest.  One warp; returns the kept count.
__device__ int compact_topk(uint64_t *buf, int na, int n, int k, uint64_t *scratch) {
  const int lane = threadIdx.x & 31;
  const int nb = n - na;
  warp_sort(buf + na, nb);
  const int keep = n < k ? n : k;
  for (int i = lane; i < na && i < keep; i += 32) {
    const int p = i + lower_bound_u64(buf + na, nb, buf[i]);
    if (p < keep) scratch[p] = buf[i];
  }
  for (int j = lane; j < nb && j < keep; j += 32) {
    const int p = j + lower_bound_u64(buf, na, buf[na + j]);
    if (p < keep) scratch[p] = buf[na + j];
  }
  __syncwarp();
  for (int i = lane; i < keep; i += 32) buf[i] = scratch[i];
  __syncwarp();
  return keep;
}
}  // namespace

int scan_query_tile(int k, int tq) { return 16 * choose(k, tq).tq; }

template <int TQ, bool TOP1>
__global__ void __launch_bounds__(THREADS) scan_f32_kernel(ScanArgs a, int cap) {
  constexpr int QT = 16 * TQ;
  constexpr int NSTAGE = nstage_for(TQ);
  extern __shared__ __align__(16) unsigned char smem[];
  float *Xs = (float *)smem;
  const size_t xbytes = (size_t)NSTAGE * XT * XROW * 4 > (size_t)NWARP * cap * 8
                            ? (size_t)NSTAGE * XT * XROW * 4
                            : (size_t)NWARP * cap * 8;
  uint64_t *s_scratch = (uint64_t *)smem;  // merge scratch, reuses the X stages between chunks
  float *Qs = (float *)(smem + xbytes);
  int32_t *s_ids = (int32_t *)(Qs + NSTAGE * QT * XROW);
  float *s_sc = (float *)(s_ids + XT);
  int32_t *s_qrow = (int32_t *)(s_sc + XT);
  int32_t *s_orow = s_qrow + QT;
  int *s_cnt = s_orow + QT;
  int *s_na = s_cnt + QT;
  uint64_t *s_tau = (uint64_t *)(((uintptr_t)(s_na + QT) + 7) & ~(uintptr_t)7);
  uint64_t *s_buf = s_tau + QT;
  __shared__ int s_tile;

  const int tid = threadIdx.x, tx = tid & 15, tq = tid >> 4;
  const int warp = tid >> 5, lane = tid & 31;
  const int nsplit = (a.tile_list && a.nsplit > 1) ? a.nsplit : 1;
  const int ntiles = a.tile_list ? *a.ntiles_dev * nsplit : (a.nq + QT - 1) / QT;
  const int nblk = (a.dims + 15) >> 4;

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_tile;
    if (item >= ntiles) break;
    const int tile = item / nsplit, range = item - tile * nsplit;
    int list, beg, cnt;
    if (a.tile_list) {
      list = a.tile_list[tile];
      beg = a.tile_beg[tile];
      cnt = a.tile_cnt[tile];
    } else {
      list = 0;
      beg = tile * QT;
      cnt = min(QT, a.nq - beg);
    }
    const int64_t moff = a.list_off[list];
    const int nl = (int)(a.list_off[list + 1] - moff);
    const float *lbase = a.xpm + moff * (int64_t)a.d_pad;
    if (tid < QT) {
      const int p = beg + tid;
      const bool v = tid < cnt;
      s_qrow[tid] = v ? (a.pair_q ? a.pair_q[p] : p) : -1;
      s_orow[tid] = v ? (a.pair_out ? a.pair_out[p] : p) : -1;
      s_cnt[tid] = 0;
      s_na[tid] = 0;
      s_tau[tid] = KEY_MAX;
    }
    __syncthreads();
    // this item's member chunks: range `range` of nsplit equal chunk ranges
    const int nchunk_all = (nl + XT - 1) / XT;
    const int cper = (nchunk_all + nsplit - 1) / nsplit;
    const int c_begin = min(nchunk_all, range * cper);
    const int nchunk = min(nchunk_all, c_begin + cper);
    for (int c = c_begin; c < nchunk; ++c) {
      const int m0 = c * XT;
      const int nm = min(XT, nl - m0);
      if (tid < XT) {
        const int m = m0 + tid;
        s_ids[tid] = tid < nm ? (a.list_ids ? a.list_ids[moff + m] : m) : 0;
        s_sc[tid] = (tid < nm && a.mscale) ? a.mscale[moff + m] : 1.f;
      }
      __syncthreads();

      auto load_stage = [&](int b, int stage) {
        const int nd4 = min(4, (a.dims - 16 * b) >> 2);
        const float *src = lbase + (int64_t)b * 16 * nl + (int64_t)m0 * 16;
        float *dst = Xs + stage * XT * XROW;
#pragma unroll
        for (int e = tid; e < XT * 4; e += THREADS) {
          const int m = e >> 2, part = e & 3;
          if (m < nm && part < nd4) cp_async16(dst + m * XROW + part * 4, src + m * 16 + part * 4);
        }
        float *qd = Qs + stage * QT * XROW;
        for (int e = tid; e < QT * 4; e += THREADS) {
          const int qi = e >> 2, part = e & 3;
          const int row = s_qrow[qi];
          if (row >= 0 && part < nd4)
            cp_async16(qd + qi * XROW + part * 4, a.qn + (int64_t)row * a.ldq + 16 * b + part * 4);
        }
      };

      float sc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) sc[i] = s_sc[tx + 16 * i];
      float acc[TQ][8];
#pragma unroll
      for (int j = 0; j < TQ; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[j][i] = 0.f;

#pragma unroll
      for (int s = 0; s < NSTAGE - 1; ++s) {
        if (s < nblk) load_stage(s, s);
        cp_async_commit();
      }
      for (int b = 0; b < nblk; ++b) {
        {
          const int bn = b + NSTAGE - 1;
          if (bn < nblk) load_stage(bn, bn % NSTAGE);
          cp_async_commit();
        }
        cp_async_wait<NSTAGE - 1>();
        __syncthreads();
        const float *xs = Xs + (b % NSTAGE) * XT * XROW;
        const float *qs = Qs + (b % NSTAGE) * QT * XROW;
        const int nd4 = min(4, (a.dims - 16 * b) >> 2);
        // FULL: every query slot of the tile is used (the batched regime);
        // otherwise slots past the tile's count are skipped
        auto step = [&](int s, auto full) {
          float4 qv[TQ], xv[8];
#pragma unroll
          for (int j = 0; j < TQ; ++j)
            qv[j] = *(const float4 *)(qs + (tq + 16 * j) * XROW + 4 * s);
#pragma unroll
          for (int i = 0; i < 8; ++i) xv[i] = *(const float4 *)(xs + (tx + 16 * i) * XROW + 4 * s);
#pragma unroll
          for (int j = 0; j < TQ; ++j) {
            if (!decltype(full)::value && tq + 16 * j >= cnt) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float t;
              t = fmaf(-sc[i], xv[i].x, qv[j].x);
              acc[j][i] = fmaf(t, t, acc[j][i]);
              t = fmaf(-sc[i], xv[i].y, qv[j].y);
              acc[j][i] = fmaf(t, t, acc[j][i]);
              t = fmaf(-sc[i], xv[i].z, qv[j].z);
              acc[j][i] = fmaf(t, t, acc[j][i]);
              t = fmaf(-sc[i], xv[i].w, qv[j].w);
              acc[j][i] = fmaf(t, t, acc[j][i]);
            }
          }
        };
        if (cnt >= QT && nd4 == 4) {
#pragma unroll
          for (int s = 0; s < 4; ++s) step(s, std::true_type{});
        } else if (cnt >= QT) {
          for (int s = 0; s < nd4; ++s) step(s, std::true_type{});
        } else if (nd4 == 4) {
#pragma unroll
          for (int s = 0; s < 4; ++s) step(s, std::false_type{});
        } else {
          for (int s = 0; s < nd4; ++s) step(s, std::false_type{});
        }
        __syncthreads();
      }

      // candidates of this chunk, appended in rounds of ROUND per query so a
      // buffer of k + ROUND keys suffices; compaction runs between rounds
      if (TOP1) {
#pragma unroll
        for (int j = 0; j < TQ; ++j) {
          const int qi = tq + 16 * j;
          if (qi < cnt) {
            const uint64_t tau = s_tau[qi];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int m = tx + 16 * i;
              if (m < nm) {
                const uint64_t key = pack_key(acc[j][i], (uint32_t)s_ids[m]);
                if (key < tau)
                  atomicMin((unsigned long long *)&s_tau[qi], (unsigned long long)key);
              }
            }
          }
        }
        __syncthreads();
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
          for (int j = 0; j < TQ; ++j) {
            const int qi = tq + 16 * j;
            if (qi < cnt) {
              const uint64_t tau = s_tau[qi];
#pragma unroll
              for (int ii = 0; ii < 2; ++ii) {
                const int m = tx + 16 * (2 * r + ii);
                if (m < nm) {
                  const uint64_t key = pack_key(acc[j][2 * r + ii], (uint32_t)s_ids[m]);
                  if (key < tau) {
                    const int pos = atomicAdd(&s_cnt[qi], 1);
                    s_buf[qi * cap + pos] = key;
                  }
                }
              }
            }
          }
          __syncthreads();
          const bool last = c == nchunk - 1 && r == 3;
          for (int qi = warp; qi < cnt; qi += NWARP) {
            const int n = s_cnt[qi];
            const int na = s_na[qi];
            if (n > cap - ROUND || (last && n > na)) {
              uint64_t *buf = s_buf + qi * cap;
              const int keep = compact_topk(buf, na, n, a.k, s_scratch + (size_t)warp * cap);
              if (lane == 0) {
                s_cnt[qi] = keep;
                s_na[qi] = keep;
                s_tau[qi] = keep == a.k ? buf[a.k - 1] : KEY_MAX;
              }
            }
          }
          __syncthreads();
        }
      }
    }
    // write the sorted per-(query, list) results
    for (int qi = warp; qi < cnt; qi += NWARP) {
      uint64_t *out = a.out_keys + ((int64_t)s_orow[qi] * nsplit + range) * a.k;
      if (TOP1) {
        if (lane == 0) out[0] = s_tau[qi];
      } else {
        const int n = s_cnt[qi];
        const uint64_t *buf = s_buf + qi * cap;
        for (int r = lane; r < a.k; r += 32) out[r] = r < n ? buf[r] : KEY_MAX;
      }
    }
    __syncthreads();
  }
}

int launch_scan_f32(const ScanArgs &a, cudaStream_t st) {
  if (a.dims % 4 != 0 || a.dims > a.d_pad || a.d_pad % 16 != 0 || a.ldq % 4 != 0 || a.k < 1)
    return fail(ADANNS_ERR_ARG, "scan: bad dimensions");
  const ScanCfg c = choose(a.k, a.tq);
  void (*kern)(ScanArgs, int) = c.cap == 0 ? scan_f32_kernel<4, true>
                                : c.tq == 4 ? scan_f32_kernel<4, false>
                                            : scan_f32_kernel<1, false>;
  // attribute and occupancy per (kernel, shared memory size), cached per device
  static std::mutex mu;
  static std::map<std::tuple<int, void *, size_t>, int> occ;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(dev, (void *)kern, c.smem);
    auto it = occ.find(key);
    // the shared-memory limit is a property of the kernel: only ever raise it
    cudaError_t e = ensure_smem((const void *)kern, c.smem);
    if (e != cudaSuccess) return cuda_fail(e, "scan attribute");
    if (it != occ.end()) {
      per_sm = it->second;
    } else {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, c.smem);
      if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      occ[key] = per_sm;
    }
  }
  const int grid = a.grid > 0 ? a.grid : num_sms() * per_sm;
  kern<<<grid, THREADS, c.smem, st>>>(a, c.cap);
  ADN_LAUNCH("scan_f32_kernel");
  return ADANNS_OK;
}

}  // namespace adn
