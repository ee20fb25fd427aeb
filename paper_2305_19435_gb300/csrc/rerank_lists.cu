// Member-major exact rerank of the shortlists (Sec. 4.3 shortlist-rerank).
//
// The B x k' shortlisted (query, member) pairs are grouped by database member
// (one counting sort over list-order member positions, so lists come out
// grouped too), so that a CTA reads each database row once from the
// prefix-major FP32 storage into shared memory and
// re-scores it against every query that shortlisted it (the query rows, far
// smaller than the database, are the gathered operand and stay in L2).  The
// exact difference-form distances are written back to the pairs' slots and a
// final per-query pass keeps the k best by (distance, id).
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {

// Pairs grouped by database member with one counting sort over the list-order
// member positions: pair e = (query e / kr, rank e % kr), given as
// (list << 32 | member position) or -1 (padding, pruned).  Its position is
// list_off[list] + member; the exclusive scan of the per-position counts is
// both the sorted order's layout and each member's first pair (mstart).
__global__ void pair_pos_kernel(const int64_t *__restrict__ cand, int64_t n,
                                const int64_t *__restrict__ list_off, int32_t *__restrict__ ppos,
                                int32_t *__restrict__ cnt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t v = cand[e];
  if (v < 0) {
    ppos[e] = -1;
    return;
  }
  const int32_t p = (int32_t)(list_off[v >> 32] + (v & 0xffffffffll));
  ppos[e] = p;
  atomicAdd(&cnt[p], 1);
}

// order[cursor[p]++] = e for every kept pair (the order among one member's
// pairs does not matter: each pair writes its own slot); npairs = the count.
// A pair's member follows from its place in the order: member p owns
// [mstart[p], mstart[p + 1]).
__global__ void pair_scatter_kernel(const int32_t *__restrict__ ppos, int64_t n,
                                    int32_t *__restrict__ cursor, int32_t *__restrict__ order,
                                    const int32_t *__restrict__ mstart, int64_t N,
                                    int64_t *__restrict__ npairs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) *npairs = mstart[N];
  if (e >= n) return;
  const int32_t p = ppos[e];
  if (p >= 0) order[atomicAdd(&cursor[p], 1)] = (int32_t)e;
}

// The pair range [first, end) of every member chunk, for this search's sort:
// a rerank CTA reads it with its chunk map entry, so that its first batch of
// pairs is requested together with the member rows
__global__ void chunk_pairs_kernel(const int4 *__restrict__ cmap, int nchunk, int mc,
                                   const int32_t *__restrict__ mstart, int2 *__restrict__ cpair) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunk) return;
  const int4 cl = cmap[c];  // (list, first member, list offset, list size)
  const int m1 = min(cl.w, cl.y + mc);
  cpair[c] = make_int2(mstart[cl.z + cl.y], mstart[cl.z + m1]);
}

// One CTA per (list, chunk of mc members): the chunk's member rows are read
// once, coalesced from the prefix-major storage, into shared memory (rows
// padded by 4 floats against bank conflicts); the chunk's pairs (consecutive
// in the sorted order) are then scored by the CTA's half-warps, each prefetching
// its next query row into registers while it scores the current one.  Only
// the query rows are gathered.  CTA i takes chunk i of the lists laid end to
// end in the index's rerank order (a nearest-neighbour chain of the
// centroids), so the CTAs resident at one time cover a few neighbouring lists
// and the query rows they gather -- those of the queries probing these lists
// -- stay in L2 while they are reused.
constexpr int RC_MAX_MC = 64;

// members per chunk: the largest of 64, 32, 16, 8 whose rows fit in 16 KB
// (at least 8), so that eight CTAs share an SM; the index keeps a chunk table
// for each of these sizes
inline int rerank_chunk_members(int d_s) {
  int mc = RC_MAX_MC;
  while (mc > 8 && mc * d_s * 4 > 16384) mc >>= 1;
  return mc;
}
static_assert(RC_MAX_MC == 64, "chunk sizes 64, 32, 16, 8 have precomputed chunk tables");

// FULL: d_s is a multiple of 512 (every half-warp lane holds 8 whole float4
// of each 512-coordinate segment), so no coordinate bound is checked.
// NT threads (a half-warp per pair in flight), at least MINB CTAs per SM: the
// query-row gathers are latency-bound, so more resident warps each holding one
// row in flight beat fewer warps double-buffering two (measured: 1.71 against
// 2.03 ms at d_s = 512, 9.25 against 10.41 ms at d_s = 2048)
template <bool FULL, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) rerank_chunks_kernel(
    const int32_t *__restrict__ order, const int32_t *__restrict__ mstart,
    const int32_t *__restrict__ list_ids, int kr,
    const float *__restrict__ qs, int ldq, int d_s, const float *__restrict__ xpm, int d_pad,
    const float *__restrict__ mscale, int mc, const int4 *__restrict__ cmap,
    const int2 *__restrict__ cpair, uint64_t *__restrict__ keys, int *__restrict__ err) {
  extern __shared__ __align__(16) float rows[];  // [mc][d_s + 4]
  constexpr int HW = NT / 16;  // half-warps per CTA
  __shared__ int s_e[NT], s_m[NT], s_q[NT];
  __shared__ float s_nu[RC_MAX_MC];
  __shared__ uint32_t s_id[RC_MAX_MC];
  __shared__ int s_ms[RC_MAX_MC + 1];  // the chunk members' first pairs, and the end
  // chunk -> (list, first member, list offset, list size): one load from the
  // index's chunk map
  const int4 cl = cmap[blockIdx.x];
  const int2 pr = cpair[blockIdx.x];
  const int64_t off = cl.z;
  const int nl = cl.w;
  const int m_first = cl.y;
  const int rs = d_s + 4, nseg = d_s >> 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = lane >> 4, hl = lane & 15, hw = warp * 2 + half;
  const unsigned hmask = half ? 0xffff0000u : 0x0000ffffu;
  // the query block is re-read by every list: keep it in L2; member rows are read once
  const uint64_t keep = l2_policy_evict_last(), stream = l2_policy_evict_first();
  {
    const int m0 = m_first;
    const int p0 = pr.x, p1 = pr.y;
    if (m0 >= nl || p0 >= p1) return;  // no pair re-scores a member of this chunk
    const int m1 = min(nl, m0 + mc), nm = m1 - m0;
    // member rows, the members' first pairs and the first batch of pairs, all
    // requested at once: block b of the chunk is nm x 16 contiguous floats
    const int per_b = nm * 4;  // float4 per block
    for (int t = threadIdx.x; t < per_b * ((d_s + 15) >> 4); t += NT) {
      const int b = t / per_b, w = t - b * per_b, mm = w >> 2, part = w & 3;
      if (4 * b + part >= nseg) continue;  // d_s = 8: half of the last block
      cp_async16_hint(rows + (size_t)mm * rs + 16 * b + 4 * part,
                      xpm + off * d_pad + (int64_t)b * 16 * nl + (int64_t)(m0 + mm) * 16 + part * 4,
                      stream);
    }
    cp_async_commit();  // the copies land while the first metadata batch loads
    const int e_first = (int)threadIdx.x < p1 - p0 ? order[p0 + threadIdx.x] : 0;
    for (int t = threadIdx.x; t <= nm; t += NT) s_ms[t] = mstart[off + m0 + t];
    for (int t = threadIdx.x; t < nm; t += NT) {
      s_nu[t] = mscale ? mscale[off + m0 + t] : 1.f;
      s_id[t] = (uint32_t)list_ids[off + m0 + t];
    }
    __syncthreads();  // s_ms visible
    for (int base = p0; base < p1; base += NT) {
      const int nb = min(NT, p1 - base);
      if (base != p0) __syncthreads();  // previous metadata consumed
      if ((int)threadIdx.x < nb) {
        const int i = base + threadIdx.x;
        const int e = base == p0 ? e_first : order[i];
        // the pair's member: the last one whose first pair is at or before i
        int lo = 0, hi = nm - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_ms[mid] <= i) lo = mid; else hi = mid - 1;
        }
        int mm = lo;
        if (e < 0 || i >= s_ms[mm + 1]) {  // inconsistent sort: report, skip the pair
          atomicOr(err, ADANNS_DEVERR_RERANK);
          mm = -1;
        }
        s_e[threadIdx.x] = max(e, 0);
        s_m[threadIdx.x] = mm;
        s_q[threadIdx.x] = max(e, 0) / kr;
      }
      cp_async_wait<0>();
      __syncthreads();  // rows and metadata visible
      // query row of pair t, first 512 coordinates, into registers
      auto load_first = [&](int t, float4(&dst)[8]) {
        const float *qr = qs + (int64_t)s_q[t] * ldq;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (FULL || hl + 16 * u < nseg)
            dst[u] = ldg_f4_hint((const float4 *)(qr + 4 * (hl + 16 * u)), keep);
      };
      // exact difference-form distance of pair t (first 512 coordinates in qv)
      auto score = [&](int t, float4(&qv)[8]) {
        const int mm = s_m[t];
        if (mm < 0) return;  // uniform in the half-warp
        const float *xr = rows + (size_t)mm * rs;
        const float nu = s_nu[mm];
        const float *qr = qs + (int64_t)s_q[t] * ldq;
        float acc = 0.f;
        for (int s0 = hl; s0 < nseg; s0 += 128) {
          if (s0 != hl) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (FULL || s0 + 16 * u < nseg)
                qv[u] = ldg_f4_hint((const float4 *)(qr + 4 * (s0 + 16 * u)), keep);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (!FULL && s0 + 16 * u >= nseg) break;
            const float4 xv = *(const float4 *)(xr + 4 * (s0 + 16 * u));
            float d;
            d = fmaf(-nu, xv.x, qv[u].x); acc = fmaf(d, d, acc);
            d = fmaf(-nu, xv.y, qv[u].y); acc = fmaf(d, d, acc);
            d = fmaf(-nu, xv.z, qv[u].z); acc = fmaf(d, d, acc);
            d = fmaf(-nu, xv.w, qv[u].w); acc = fmaf(d, d, acc);
          }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(hmask, acc, o);
        if (hl == 0) keys[s_e[t]] = pack_key(acc, s_id[mm]);
      };
      // the half-warp's pairs t = hw, hw + HW, ...
      float4 qa[8];
      for (int t = hw; t < nb; t += HW) {
        load_first(t, qa);
        score(t, qa);
      }
    }
  }
}

// Ascending bitonic sort of 256 keys held 8 per lane (lane l holds positions
// 8l .. 8l + 7): strides below 8 compare within a lane, larger ones across
// lanes by shuffles; the direction of each compare-exchange is that of the
// block of `size` positions holding it (ascending for even blocks).
__device__ __forceinline__ void warp_sort256(uint64_t (&v)[8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 256; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 8) {
        const int ls = stride >> 3;
        const bool lower = (lane & ls) == 0;
        const bool asc = ((lane * 8) & size) == 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint64_t o = __shfl_xor_sync(0xffffffffu, v[j], ls);
          const uint64_t lo = o < v[j] ? o : v[j], hi = o < v[j] ? v[j] : o;
          v[j] = lower == asc ? lo : hi;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j & stride) continue;
          const bool asc = ((lane * 8 + j) & size) == 0;
          const uint64_t a = v[j], b = v[j | stride];
          const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
          v[j] = asc ? lo : hi;
          v[j | stride] = asc ? hi : lo;
        }
      }
    }
  }
}

// per query (one warp): sort its kr keys, write the k best
__global__ void final_topk_kernel(const uint64_t *__restrict__ keys, int kr, int64_t B, int k,
                                  int64_t *__restrict__ out_ids, float *__restrict__ out_dist) {
  extern __shared__ uint64_t kb[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * 4 + warp;
  if (q >= B) return;
  uint64_t *buf = kb + (size_t)warp * kr;
  // keep only the re-scored slots (pruned and padding slots hold the empty key)
  int n = 0;
  for (int r0 = 0; r0 < kr; r0 += 128) {
    uint64_t key[4];  // four loads in flight before the first ballot
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + 32 * u + lane;
      key[u] = r < kr ? __ldg(keys + q * kr + r) : KEY_MAX;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned m = __ballot_sync(0xffffffffu, key[u] != KEY_MAX);
      if (key[u] != KEY_MAX) buf[n + __popc(m & lanemask_lt())] = key[u];
      n += __popc(m);
    }
  }
  __syncwarp();
  if (n <= 256) {
    // the common case (pruned shortlists): sorted in registers
    uint64_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = lane * 8 + j;
      v[j] = r < n ? buf[r] : KEY_MAX;
    }
    warp_sort256(v);
    // back through shared memory (the first min(k, 256) positions, k <= kr), so
    // that the results leave as whole rows: lanes write consecutive entries
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (lane * 8 + j < k) buf[lane * 8 + j] = v[j];
    __syncwarp();
    for (int r = lane; r < k; r += 32) {
      const uint64_t key = r < 256 ? buf[r] : KEY_MAX;  // k above 256: padding
      out_ids[q * k + r] = key == KEY_MAX ? -1 : (int64_t)(uint32_t)(key & 0xffffffffu);
      out_dist[q * k + r] = key == KEY_MAX ? __int_as_float(0x7f800000)
                                           : __uint_as_float((uint32_t)(key >> 32));
    }
    return;
  }
  warp_sort(buf, n);
  for (int r = lane; r < k; r += 32) {
    const uint64_t key = r < n ? buf[r] : KEY_MAX;
    out_ids[q * k + r] = key == KEY_MAX ? -1 : (int64_t)(uint32_t)(key & 0xffffffffu);
    out_dist[q * k + r] = key == KEY_MAX ? __int_as_float(0x7f800000)
                                         : __uint_as_float((uint32_t)(key >> 32));
  }
}

// per query: the k best of kr packed keys, as (ids, distances)
int launch_final_topk(const uint64_t *keys, int kr, int64_t B, int k, int64_t *out_ids,
                      float *out_dist, cudaStream_t st) {
  if (B <= 0) return ADANNS_OK;
  const size_t fs = (size_t)4 * kr * 8;
  ADN_CUDA(ensure_smem((const void *)final_topk_kernel, fs));
  final_topk_kernel<<<(unsigned)((B + 3) / 4), 128, fs, st>>>(keys, kr, B, k, out_ids, out_dist);
  ADN_LAUNCH("final_topk_kernel");
  return ADANNS_OK;
}

int launch_rerank_lists(const int64_t *cand, int kr, int64_t B, const float *qs, int ldq, int d_s,
                        const adanns_index *idx, const float *mscale, int k, int64_t *out_ids,
                        float *out_dist, cudaStream_t st) {
  if (B <= 0) return ADANNS_OK;
  const int64_t n = B * kr;
  if (n > INT32_MAX) return fail(ADANNS_ERR_ARG, "rerank slice too large");
  const int64_t N = idx->N;
  Scratch s(st);
  int32_t *ppos, *order, *mstart, *cursor;
  int2 *cpair;
  int64_t *npairs;
  uint64_t *keys;
  int rc;
  if ((rc = s.get(&ppos, n)) || (rc = s.get(&order, n)) ||
      (rc = s.get(&keys, n)) || (rc = s.get(&mstart, (size_t)N + 1)) ||
      (rc = s.get(&cursor, (size_t)N + 1)) || (rc = s.get(&npairs, 1)))
    return rc;
  const int mc = rerank_chunk_members(d_s);
  const int ci = rerank_chunk_index(mc);
  const int chunks = idx->rr_chunks[ci];
  if ((rc = s.get(&cpair, (size_t)std::max(chunks, 1)))) return rc;
  {
    StageTimer t(ST_RR_SORT, st);
    ADN_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (N + 1), st));
    pair_pos_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cand, n, idx->list_off, ppos,
                                                                  cursor);
    ADN_LAUNCH("pair_pos_kernel");
    if ((rc = launch_scan_i32(cursor, N + 1, mstart, st))) return rc;
    ADN_CUDA(cudaMemcpyAsync(cursor, mstart, sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToDevice,
                             st));
    pair_scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ppos, n, cursor, order, mstart,
                                                                      N, npairs);
    ADN_LAUNCH("pair_scatter_kernel");
    if (chunks > 0) {
      chunk_pairs_kernel<<<(unsigned)((chunks + 255) / 256), 256, 0, st>>>(
          idx->rr_cmap[ci], chunks, mc, mstart, cpair);
      ADN_LAUNCH("chunk_pairs_kernel");
    }
  }
  profile_count(PC_RERANK_PAIRS, npairs, st);  // pairs left after pruning
  profile_count_host(PC_SHORTLIST_SLOTS, n);
  {
    StageTimer t(ST_RR_PAIRS, st);
    const size_t rs = (size_t)mc * (d_s + 4) * 4;
    const bool full = d_s % 512 == 0;
    // slots of padding or pruned candidates keep the empty key
    ADN_CUDA(cudaMemsetAsync(keys, 0xFF, sizeof(uint64_t) * n, st));
    if (chunks > 0) {
      // long prefixes (eight-member chunks of up to 64 KB of rows): 256 threads
      // share a chunk; shorter ones: 128 threads, eight CTAs per SM
      auto go = [&](auto kern, int nt) -> cudaError_t {
        cudaError_t e = ensure_smem((const void *)kern, rs);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)chunks, nt, rs, st>>>(order, mstart, idx->list_ids, kr, qs, ldq,
                                               d_s, idx->xpm, idx->d_pad, mscale, mc,
                                               idx->rr_cmap[ci], cpair, keys, idx->dev_err);
        return cudaSuccess;
      };
      const bool wide = d_s >= 1024;
      cudaError_t e;
      if (full)
        e = wide ? go(rerank_chunks_kernel<true, 256, 4>, 256)
                 : go(rerank_chunks_kernel<true, 128, 8>, 128);
      else
        e = wide ? go(rerank_chunks_kernel<false, 256, 4>, 256)
                 : go(rerank_chunks_kernel<false, 128, 8>, 128);
      if (e != cudaSuccess) return cuda_fail(e, "rerank attribute");
      ADN_LAUNCH("rerank_chunks_kernel");
    }
  }
  {
    StageTimer t(ST_RR_FINAL, st);
    const size_t fs = (size_t)4 * kr * 8;
    ADN_CUDA(ensure_smem((const void *)final_topk_kernel, (size_t)(fs)));
    final_topk_kernel<<<(unsigned)((B + 3) / 4), 128, fs, st>>>(keys, kr, B, k, out_ids, out_dist);
    ADN_LAUNCH("final_topk_kernel");
  }
  return ADANNS_OK;
}

}  // namespace adn
