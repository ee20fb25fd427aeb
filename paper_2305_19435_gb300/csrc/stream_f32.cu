// Exact FP32 list scan for the memory-bound regime: few queries probe each
// list (Algorithm 1 linear scan when the batch is small against nlist), so a
// member row is used by a handful of queries and the scan is a stream of the
// probed lists' d_s prefixes.
//
// Work unit = (probe tile, chunk of 256 members, group of up to 4 of the
// tile's queries): units cost about the same whatever the list's popularity,
// and are enumerated by an exclusive scan of each tile's unit count.  One
// thread per member: the member's 16-coordinate prefix blocks are read with
// 16-byte loads straight into registers (a warp covers 32 consecutive
// members, 2 KB contiguous per block in the prefix-major layout), the next
// block in flight while one is used, and the distances to the group's
// queries accumulate in registers; no barrier inside the stream.  The
// arithmetic is the FP32 scan's (t = q_j - s_x x_j, acc += t * t over j
// ascending), so the distances are bit-identical to it; each one is written
// as FP32 bits into the query's candidate segment, and select32_kernel then
// keeps the k best by (distance, id).
//
// A batch of queries with their own budgets (d_s, nprobe, k per query) runs
// as one launch of each kernel: masked probe slots make no pairs, a unit
// streams its member rows up to the largest d_s of its queries while each
// query stops accumulating at its own d_s (with its own per-member scale at
// that prefix), and the selection keeps the batch's largest k, of which a
// query's own k results are the prefix.
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {
namespace {

constexpr int SF_THREADS = 256;  // one chunk of members per work unit
constexpr int SF_QT = 16;        // queries per probe tile
constexpr int SF_QG = 4;         // queries per work unit

struct StreamArgs {
  const float *xpm;  // prefix-major FP32 lists
  int d_pad, dims;
  const int64_t *list_off;
  const float *mscale;  // per-member scale (inverse prefix norm), or null
  const float *qn;      // prepared query rows
  int ldq;
  // per-query prefixes (or null: every query scans a.dims): d_s of each query
  // and the index's inverse prefix norms [granularity][N] with each query's
  // granularity index (null with the raw metric)
  const int32_t *qds, *qgi;
  const float *invn;
  int64_t N;
  const int32_t *tile_list, *tile_beg, *tile_cnt;
  const int *ntiles_dev;
  const int64_t *uoff;  // first work unit of each tile (exclusive scan of its units)
  const int64_t *nunits;
  const int32_t *pair_q, *pair_out;
  const int64_t *pbase;  // candidate segment start of each (query, probe) pair
  uint32_t *cand;
  int *counter;
};

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg((const float4 *)p); }

// units of a tile: member chunks x query groups (0 past the tile count)
__global__ void stream_units_kernel(const int32_t *__restrict__ tl, const int32_t *__restrict__ tc,
                                    const int *__restrict__ ntiles, const int64_t *__restrict__ list_off,
                                    int64_t max_tiles, int64_t *__restrict__ units) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= max_tiles) return;
  int64_t u = 0;
  if (t < *ntiles) {
    const int l = tl[t];
    const int64_t npad = (list_off[l + 1] - list_off[l] + 7) & ~7ll;
    u = ((npad + SF_THREADS - 1) / SF_THREADS) * ((tc[t] + SF_QG - 1) / SF_QG);
  }
  units[t] = u;
}

// acc[j] += sum over the block's coordinates (nd4 groups of 4) of (q - s x)^2
template <bool FULL>
__device__ __forceinline__ void block_step(float (&acc)[SF_QG], const float4 (&x)[4], float sc,
                                           const float *const *qrow, int cnt, int off, int nd4) {
#pragma unroll
  for (int j = 0; j < SF_QG; ++j) {
    if (j >= cnt) break;
    const float *qb = qrow[j] + off;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (!FULL && s >= nd4) break;
      const float4 q = ldg4(qb + 4 * s);
      float t;
      t = fmaf(-sc, x[s].x, q.x);
      acc[j] = fmaf(t, t, acc[j]);
      t = fmaf(-sc, x[s].y, q.y);
      acc[j] = fmaf(t, t, acc[j]);
      t = fmaf(-sc, x[s].z, q.z);
      acc[j] = fmaf(t, t, acc[j]);
      t = fmaf(-sc, x[s].w, q.w);
      acc[j] = fmaf(t, t, acc[j]);
    }
  }
}

// The same for a group whose queries stop at their own prefixes: query j
// takes the block's coordinates below ds[j] (multiples of 4), scaled by its
// own sc[j].
__device__ __forceinline__ void block_step_var(float (&acc)[SF_QG], const float4 (&x)[4],
                                               const float (&sc)[SF_QG],
                                               const float *const *qrow, const int (&ds)[SF_QG],
                                               int cnt, int off) {
#pragma unroll
  for (int j = 0; j < SF_QG; ++j) {
    if (j >= cnt) break;
    const int nd4 = min(4, (ds[j] - off) >> 2);
    const float *qb = qrow[j] + off;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (s >= nd4) break;
      const float4 q = ldg4(qb + 4 * s);
      float t;
      t = fmaf(-sc[j], x[s].x, q.x);
      acc[j] = fmaf(t, t, acc[j]);
      t = fmaf(-sc[j], x[s].y, q.y);
      acc[j] = fmaf(t, t, acc[j]);
      t = fmaf(-sc[j], x[s].z, q.z);
      acc[j] = fmaf(t, t, acc[j]);
      t = fmaf(-sc[j], x[s].w, q.w);
      acc[j] = fmaf(t, t, acc[j]);
    }
  }
}

// Per-query prefixes: units as in dist_f32_kernel; a unit's member rows are
// streamed to the largest d_s of its queries.
__global__ void __launch_bounds__(SF_THREADS, 4) dist_f32_var_kernel(StreamArgs a) {
  __shared__ int s_item;
  __shared__ const float *s_qp[SF_QG];
  __shared__ const float *s_sp[SF_QG];  // each query's per-member scales (or null)
  __shared__ int64_t s_pb[SF_QG];
  __shared__ int s_ds[SF_QG];
  const int tid = threadIdx.x;
  const int64_t nunits = *a.nunits;
  const int ntiles = *a.ntiles_dev;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= nunits) break;
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.uoff[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int tile = lo;
    const int list = a.tile_list[tile], beg = a.tile_beg[tile], tcnt = a.tile_cnt[tile];
    const int ngrp = (tcnt + SF_QG - 1) / SF_QG;
    const int u = (int)(item - a.uoff[tile]);
    const int chunk = u / ngrp, g = u - chunk * ngrp;
    const int q0 = g * SF_QG, cnt = min(SF_QG, tcnt - q0);
    if (tid < cnt) {
      const int q = a.pair_q[beg + q0 + tid];
      s_qp[tid] = a.qn + (int64_t)q * a.ldq;
      s_pb[tid] = a.pbase[a.pair_out[beg + q0 + tid]];
      s_ds[tid] = a.qds[q];
      s_sp[tid] = a.invn ? a.invn + (int64_t)a.qgi[q] * a.N : nullptr;
    }
    __syncthreads();
    const int64_t moff = a.list_off[list];
    const int nl = (int)(a.list_off[list + 1] - moff), npad = (nl + 7) & ~7;
    const int m = chunk * SF_THREADS + tid;
    if (m < nl) {
      int ds[SF_QG], dmax = 0;
      float sc[SF_QG];
#pragma unroll
      for (int j = 0; j < SF_QG; ++j) {
        ds[j] = j < cnt ? s_ds[j] : 0;
        sc[j] = j < cnt && s_sp[j] ? __ldg(s_sp[j] + moff + m) : 1.f;
        dmax = max(dmax, ds[j]);
      }
      const int nblk = (dmax + 15) >> 4;
      const float *xr = a.xpm + moff * (int64_t)a.d_pad + (int64_t)m * 16;
      const int64_t bstride = (int64_t)16 * nl;
      const float *const *qrow = s_qp;
      float acc[SF_QG];
#pragma unroll
      for (int j = 0; j < SF_QG; ++j) acc[j] = 0.f;
      float4 xa[4], xb[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) xa[s] = ldg4(xr + 4 * s);
      int b = 0;
      for (; b + 2 <= nblk; b += 2) {
#pragma unroll
        for (int s = 0; s < 4; ++s) xb[s] = ldg4(xr + (b + 1) * bstride + 4 * s);
        block_step_var(acc, xa, sc, qrow, ds, cnt, 16 * b);
        if (b + 2 < nblk) {
#pragma unroll
          for (int s = 0; s < 4; ++s) xa[s] = ldg4(xr + (b + 2) * bstride + 4 * s);
        }
        block_step_var(acc, xb, sc, qrow, ds, cnt, 16 * (b + 1));
      }
      if (b < nblk) block_step_var(acc, xa, sc, qrow, ds, cnt, 16 * b);
#pragma unroll
      for (int j = 0; j < SF_QG; ++j)
        if (j < cnt) a.cand[s_pb[j] + m] = __float_as_uint(acc[j]);
    } else if (m < npad) {
      for (int j = 0; j < cnt; ++j) a.cand[s_pb[j] + m] = 0xFFFFFFFFu;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SF_THREADS, 4) dist_f32_kernel(StreamArgs a) {
  __shared__ int s_item;
  __shared__ const float *s_qp[SF_QG];  // the unit's query rows
  __shared__ int64_t s_pb[SF_QG];
  const int tid = threadIdx.x;
  const int64_t nunits = *a.nunits;
  const int ntiles = *a.ntiles_dev;
  const int nblk = (a.dims + 15) >> 4;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= nunits) break;
    // the tile holding this unit: the last tile whose first unit is <= item
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.uoff[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int tile = lo;
    const int list = a.tile_list[tile], beg = a.tile_beg[tile], tcnt = a.tile_cnt[tile];
    const int ngrp = (tcnt + SF_QG - 1) / SF_QG;
    const int u = (int)(item - a.uoff[tile]);
    const int chunk = u / ngrp, g = u - chunk * ngrp;
    const int q0 = g * SF_QG, cnt = min(SF_QG, tcnt - q0);
    if (tid < cnt) {
      s_qp[tid] = a.qn + (int64_t)a.pair_q[beg + q0 + tid] * a.ldq;
      s_pb[tid] = a.pbase[a.pair_out[beg + q0 + tid]];
    }
    __syncthreads();
    const int64_t moff = a.list_off[list];
    const int nl = (int)(a.list_off[list + 1] - moff), npad = (nl + 7) & ~7;
    const int m = chunk * SF_THREADS + tid;
    if (m < nl) {
      const float sc = a.mscale ? __ldg(a.mscale + moff + m) : 1.f;
      const float *xr = a.xpm + moff * (int64_t)a.d_pad + (int64_t)m * 16;
      const int64_t bstride = (int64_t)16 * nl;
      const float *const *qrow = s_qp;
      float acc[SF_QG];
#pragma unroll
      for (int j = 0; j < SF_QG; ++j) acc[j] = 0.f;
      float4 xa[4], xb[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) xa[s] = ldg4(xr + 4 * s);
      int b = 0;
      // two blocks per trip: the next block loads while this one is used
      for (; b + 2 <= nblk; b += 2) {
#pragma unroll
        for (int s = 0; s < 4; ++s) xb[s] = ldg4(xr + (b + 1) * bstride + 4 * s);
        block_step<true>(acc, xa, sc, qrow, cnt, 16 * b, 4);
        if (b + 2 < nblk) {
#pragma unroll
          for (int s = 0; s < 4; ++s) xa[s] = ldg4(xr + (b + 2) * bstride + 4 * s);
        }
        const int nd4b = min(4, (a.dims - 16 * (b + 1)) >> 2);
        if (nd4b == 4) block_step<true>(acc, xb, sc, qrow, cnt, 16 * (b + 1), 4);
        else block_step<false>(acc, xb, sc, qrow, cnt, 16 * (b + 1), nd4b);
      }
      if (b < nblk) {  // odd block count: the last block is in xa
        const int nd4 = min(4, (a.dims - 16 * b) >> 2);
        if (nd4 == 4) block_step<true>(acc, xa, sc, qrow, cnt, 16 * b, 4);
        else block_step<false>(acc, xa, sc, qrow, cnt, 16 * b, nd4);
      }
#pragma unroll
      for (int j = 0; j < SF_QG; ++j)
        if (j < cnt) a.cand[s_pb[j] + m] = __float_as_uint(acc[j]);
    } else if (m < npad) {  // the segment's padding
      for (int j = 0; j < cnt; ++j) a.cand[s_pb[j] + m] = 0xFFFFFFFFu;
    }
    __syncthreads();  // s_qp / s_pb are rewritten by the next unit
  }
}

}  // namespace

// Few queries per probed list: prefer the streaming scan (ADANNS_OPT_FP32_STREAM = 0
// keeps the shared-memory tiled scan everywhere)
bool fp32_stream_enabled(double queries_per_list, int nprobe, int k, int d_s) {
  if (!option(ADANNS_OPT_FP32_STREAM) || nprobe > 256) return false;
  const int t = k > 0 ? tuned_scan_tq(k, d_s, queries_per_list) : 0;
  if (t != 0) return t == TUNE_STREAM;
  return queries_per_list <= 16.0;
}

int search_f32_stream(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                      int nprobe, int k, int64_t *out_ids, float *out_dist, int32_t *out_probes,
                      cudaStream_t st, const QueryBudgets *qb) {
  const int nlist = idx->nlist;
  const int dcp = pad16(d_c), dsp = pad16(d_s);
  const int64_t seg_q = max_probe_members(idx, nprobe);
  const int64_t per_q =
      seg_q * 4 + (int64_t)(dcp + dsp) * 4 + (int64_t)k * 8 + (int64_t)nprobe * 40 + 16;
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, scratch_budget() / per_q));
  const int64_t max_tiles = (Bc * nprobe + SF_QT - 1) / SF_QT + nlist;
  Scratch s(st);
  float *qc, *qs;
  uint64_t *ckeys, *keys;
  uint32_t *cand;
  int64_t *qtot, *qbase, *pbase, *units, *uoff, *nunits;
  int32_t *lcnt, *lbeg, *lfill, *tbeg, *pair_q, *pair_out, *tl, *tb, *tc;
  int *ntiles, *counter;
  int rc;
  if ((rc = s.get(&qc, (size_t)Bc * dcp)) || (rc = s.get(&qs, (size_t)Bc * dsp)) ||
      (rc = s.get(&ckeys, (size_t)Bc * nprobe)) || (rc = s.get(&cand, (size_t)(Bc * seg_q))) ||
      (rc = s.get(&keys, (size_t)Bc * k)) || (rc = s.get(&qtot, (size_t)Bc)) ||
      (rc = s.get(&qbase, (size_t)Bc)) || (rc = s.get(&pbase, (size_t)Bc * nprobe)) ||
      (rc = s.get(&lcnt, nlist)) || (rc = s.get(&lbeg, nlist)) || (rc = s.get(&lfill, nlist)) ||
      (rc = s.get(&tbeg, nlist)) || (rc = s.get(&pair_q, (size_t)Bc * nprobe)) ||
      (rc = s.get(&pair_out, (size_t)Bc * nprobe)) || (rc = s.get(&tl, max_tiles)) ||
      (rc = s.get(&tb, max_tiles)) || (rc = s.get(&tc, max_tiles)) || (rc = s.get(&ntiles, 1)) ||
      (rc = s.get(&counter, 2)) || (rc = s.get(&units, max_tiles)) ||
      (rc = s.get(&uoff, max_tiles)) || (rc = s.get(&nunits, 1)))
    return rc;
  const float *mscale = idx->metric == ADANNS_METRIC_L2_PREFIXNORM
                            ? idx->invn + (int64_t)gran_index(d_s) * idx->N
                            : nullptr;
  for (int64_t b0 = 0; b0 < B; b0 += Bc) {
    const int64_t nb = std::min(Bc, B - b0);
    const QueryBudgets bq = qb ? qb->at(b0) : QueryBudgets{};
    {
      StageTimer t(ST_PREP, st);
      if ((rc = launch_prep_queries(queries + b0 * idx->d, nb, idx->d, d_c, d_s, idx->metric, qc,
                                    dcp, qs, dsp, st, bq.ds)))
        return rc;
    }
    ADN_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st));
    {
      StageTimer t(ST_COARSE, st);
      if ((rc = run_coarse(idx, qc, dcp, nb, d_c, nprobe, ckeys, counter, st))) return rc;
      if ((rc = launch_mask_probes(ckeys, nb, nprobe, bq.np, st))) return rc;
    }
    {
      StageTimer t(ST_INVERT, st);
      if ((rc = launch_invert_probes(ckeys, nb, nprobe, nlist, SF_QT, lcnt, lbeg, lfill, tbeg,
                                     pair_q, pair_out, tl, tb, tc, ntiles,
                                     out_probes ? out_probes + b0 * nprobe : nullptr, st)))
        return rc;
      if ((rc = launch_cand_segments(ckeys, nb, nprobe, idx->list_off, qtot, qbase, pbase, st)))
        return rc;
    }
    {
      StageTimer t(ST_SCAN, st);
      stream_units_kernel<<<(unsigned)((max_tiles + 255) / 256), 256, 0, st>>>(
          tl, tc, ntiles, idx->list_off, max_tiles, units);
      ADN_LAUNCH("stream_units_kernel");
      if ((rc = launch_scan64(units, max_tiles, uoff, nunits, st))) return rc;
      StreamArgs a{};
      a.xpm = idx->xpm;
      a.d_pad = idx->d_pad;
      a.dims = d_s;
      a.list_off = idx->list_off;
      a.mscale = mscale;
      a.qn = qs;
      a.ldq = dsp;
      a.tile_list = tl;
      a.tile_beg = tb;
      a.tile_cnt = tc;
      a.ntiles_dev = ntiles;
      a.uoff = uoff;
      a.nunits = nunits;
      a.pair_q = pair_q;
      a.pair_out = pair_out;
      a.pbase = pbase;
      a.cand = cand;
      a.counter = counter + 1;
      a.qds = bq.ds;
      a.qgi = bq.gi;
      a.invn = idx->metric == ADANNS_METRIC_L2_PREFIXNORM ? idx->invn : nullptr;
      a.N = idx->N;
      auto kern = bq.ds ? dist_f32_var_kernel : dist_f32_kernel;
      int per_sm = 1;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SF_THREADS, 0) !=
              cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      kern<<<num_sms() * per_sm, SF_THREADS, 0, st>>>(a);
      ADN_LAUNCH(bq.ds ? "dist_f32_var_kernel" : "dist_f32_kernel");
    }
    {
      StageTimer t(ST_MERGE, st);
      if ((rc = launch_select32(cand, ckeys, nprobe, qbase, idx->list_off, idx->list_ids, nb, k,
                                keys, st)))
        return rc;
      if ((rc = launch_final_topk(keys, k, nb, k, out_ids + b0 * k, out_dist + b0 * k, st)))
        return rc;
      if ((rc = launch_pad_rows(out_ids + b0 * k, out_dist + b0 * k, nb, k, bq.k, st))) return rc;
    }
  }
  return ADANNS_OK;
}

}  // namespace adn
