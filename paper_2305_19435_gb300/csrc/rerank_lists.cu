// Member-major exact rerank of the shortlists (Sec. 4.3 shortlist-rerank).
//
// The B x k' shortlisted (query, member) pairs are grouped by list (stable
// counting sort) and, inside each list, by member, so that a warp reads each
// database row once from the prefix-major FP32 storage into shared memory and
// re-scores it against every query that shortlisted it (the query rows, far
// smaller than the database, are the gathered operand and stay in L2).  The
// exact difference-form distances are written back to the pairs' slots and a
// final per-query pass keeps the k best by (distance, id).
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {

// pair e = (query e / kr, rank e % kr): its list (nlist for padding) and member index
__global__ void pair_lists_kernel(const int64_t *__restrict__ cand, int64_t n, int nlist,
                                  const int32_t *__restrict__ assign,
                                  const int32_t *__restrict__ pos,
                                  const int64_t *__restrict__ list_off, int32_t *__restrict__ plist,
                                  int32_t *__restrict__ pmem) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t id = cand[e];
  if (id < 0) {
    plist[e] = nlist;
    pmem[e] = 0;
    return;
  }
  const int l = assign[id];
  plist[e] = l;
  pmem[e] = (int32_t)(pos[id] - list_off[l]);
}

// one CTA per list group: reorder that group's pairs by member index
__global__ void member_sort_kernel(const int64_t *__restrict__ goff, const int32_t *__restrict__ byl,
                                   const int32_t *__restrict__ pmem,
                                   const int64_t *__restrict__ list_off, int nlist,
                                   int32_t *__restrict__ out) {
  extern __shared__ int hist[];
  const int l = blockIdx.x;
  const int64_t lo = goff[l], hi = goff[l + 1];
  const int nm = l < nlist ? (int)(list_off[l + 1] - list_off[l]) : 1;
  for (int i = threadIdx.x; i <= nm; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&hist[pmem[byl[i]] + 1], 1);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i <= nm; ++i) hist[i] += hist[i - 1];
  __syncthreads();
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int e = byl[i];
    const int p = atomicAdd(&hist[pmem[e]], 1);
    out[lo + p] = e;
  }
}

// A warp walks 32 consecutive sorted pairs, two at a time (one per half-warp,
// so two query rows are in flight); each half keeps its current member row
// in its own shared buffer and reloads it only when its member changes.
constexpr int RL_WARPS = 8;

__global__ void __launch_bounds__(RL_WARPS * 32) rerank_pairs_kernel(
    const int32_t *__restrict__ order, int64_t npairs, const int32_t *__restrict__ plist,
    const int32_t *__restrict__ pmem, const int64_t *__restrict__ cand, int kr,
    const float *__restrict__ qs, int ldq, int d_s, const float *__restrict__ xpm, int d_pad,
    const int64_t *__restrict__ list_off, const float *__restrict__ mscale, int nlist,
    uint64_t *__restrict__ keys) {
  extern __shared__ __align__(16) float rowbuf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = lane >> 4, hl = lane & 15;
  const unsigned hmask = half ? 0xffff0000u : 0x0000ffffu;
  float *row = rowbuf + ((size_t)warp * 2 + half) * d_s;
  const int64_t w0 = ((int64_t)blockIdx.x * RL_WARPS + warp) * 32;
  if (w0 >= npairs) return;
  const int64_t w1 = min(npairs, w0 + 32);
  int cur_l = -1, cur_m = -1;
  float nu = 1.f;
  const int nseg = d_s >> 2;
  for (int64_t i = w0 + half; i < w1; i += 2) {
    const int e = order[i];
    const int l = plist[e];
    if (l >= nlist) {
      if (hl == 0) keys[e] = KEY_MAX;
      continue;
    }
    const int m = pmem[e];
    if (l != cur_l || m != cur_m) {
      const int64_t off = list_off[l];
      const int64_t nl = list_off[l + 1] - off;
      const float *base = xpm + off * d_pad + (int64_t)m * 16;
      __syncwarp(hmask);
      for (int s = hl; s < nseg; s += 16) {
        const int b = s >> 2, part = s & 3;
        *(float4 *)(row + 4 * s) = *(const float4 *)(base + (int64_t)b * 16 * nl + part * 4);
      }
      nu = mscale ? mscale[off + m] : 1.f;
      cur_l = l;
      cur_m = m;
      __syncwarp(hmask);
    }
    const int64_t q = e / kr;
    const float *qr = qs + q * ldq;
    float acc = 0.f;
    for (int s0 = hl; s0 < nseg; s0 += 128) {
      float4 qv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + 16 * u < nseg) qv[u] = __ldg((const float4 *)(qr + 4 * (s0 + 16 * u)));
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (s0 + 16 * u >= nseg) break;
        const float4 xv = *(const float4 *)(row + 4 * (s0 + 16 * u));
        float t;
        t = fmaf(-nu, xv.x, qv[u].x); acc = fmaf(t, t, acc);
        t = fmaf(-nu, xv.y, qv[u].y); acc = fmaf(t, t, acc);
        t = fmaf(-nu, xv.z, qv[u].z); acc = fmaf(t, t, acc);
        t = fmaf(-nu, xv.w, qv[u].w); acc = fmaf(t, t, acc);
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(hmask, acc, o);
    if (hl == 0) keys[e] = pack_key(acc, (uint32_t)cand[e]);
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
  for (int r = lane; r < kr; r += 32) buf[r] = keys[q * kr + r];
  __syncwarp();
  warp_sort(buf, kr);
  for (int r = lane; r < k; r += 32) {
    const uint64_t key = r < kr ? buf[r] : KEY_MAX;
    out_ids[q * k + r] = key == KEY_MAX ? -1 : (int64_t)(uint32_t)(key & 0xffffffffu);
    out_dist[q * k + r] = key == KEY_MAX ? __int_as_float(0x7f800000)
                                         : __uint_as_float((uint32_t)(key >> 32));
  }
}

int launch_rerank_lists(const int64_t *cand, int kr, int64_t B, const float *qs, int ldq, int d_s,
                        const adanns_index *idx, const float *mscale, int k, int64_t *out_ids,
                        float *out_dist, cudaStream_t st) {
  if (B <= 0) return ADANNS_OK;
  const int64_t n = B * kr;
  if (n > INT32_MAX) return fail(ADANNS_ERR_ARG, "rerank slice too large");
  const int nlist = idx->nlist;
  Scratch s(st);
  int32_t *plist, *pmem, *byl, *order;
  int64_t *goff;
  uint64_t *keys;
  int rc;
  if ((rc = s.get(&plist, n)) || (rc = s.get(&pmem, n)) || (rc = s.get(&byl, n)) ||
      (rc = s.get(&order, n)) || (rc = s.get(&goff, (size_t)nlist + 2)) || (rc = s.get(&keys, n)))
    return rc;
  {
    StageTimer t(ST_RR_SORT, st);
    pair_lists_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        cand, n, nlist, idx->assign, idx->pos_of_id, idx->list_off, plist, pmem);
    ADN_LAUNCH("pair_lists_kernel");
    if ((rc = build_csr(plist, n, nlist + 1, goff, byl, st))) return rc;
    const size_t hs = ((size_t)idx->max_list + 2) * 4;
    ADN_CUDA(ensure_smem((const void *)member_sort_kernel, (size_t)(hs)));
    member_sort_kernel<<<nlist + 1, 256, hs, st>>>(goff, byl, pmem, idx->list_off, nlist, order);
    ADN_LAUNCH("member_sort_kernel");
  }
  {
    StageTimer t(ST_RR_PAIRS, st);
    const size_t rs = (size_t)RL_WARPS * 2 * d_s * 4;
    ADN_CUDA(ensure_smem((const void *)rerank_pairs_kernel, (size_t)(rs)));
    const int64_t warps = (n + 31) / 32;
    rerank_pairs_kernel<<<(unsigned)((warps + RL_WARPS - 1) / RL_WARPS), RL_WARPS * 32, rs, st>>>(
        order, n, plist, pmem, cand, kr, qs, ldq, d_s, idx->xpm, idx->d_pad, idx->list_off,
        mscale, nlist, keys);
    ADN_LAUNCH("rerank_pairs_kernel");
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
