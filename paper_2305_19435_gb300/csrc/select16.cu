// Per-query shortlist of the mixed-precision search (Sec. 4.3 shortlist): the
// kk smallest 16-bit keys (fixed-point approximate distances) of the query's
// candidate region [qbase, qbase + ptotal) (probed lists in rank order, each
// padded to 8 with the largest key).  One warp per query, four per CTA, no
// block barriers, so many queries' memory latencies overlap on an SM:
//  1. a sample of up to 2,048 keys (256 evenly spaced 16-byte runs) gives a
//     threshold T aimed at (kk + SW_BUF) / 2 smaller keys (radix select on
//     the sample);
//  2. one pass over the region (twelve 16-byte loads in flight per lane)
//     compacts every key < T, with its position, into a per-warp buffer;
//  3. if the buffer holds between kk and SW_BUF keys, an exact two-digit
//     radix select on it fixes the cut; otherwise the same select runs over
//     the whole region in position order.
// Keys equal to the cut are taken in candidate-position order (list rank,
// then member position), independent of thread timing.  With certified
// pruning, winners whose key exceeds the k-th smallest key by more than the
// query's delta are written as -1 (the bound is derived beside
// shortlist_prune_enabled).  A winner is written as (list << 32 | member
// position); padding slots as -1.
#include "devutil.cuh"
#include "internal.cuh"

namespace adn {
namespace {

constexpr int SW_WARPS = 4;
constexpr int SW_SAMPLE = 2048;
constexpr int SW_BUF = 1024;
constexpr int SW_TIE = 128;
constexpr int SW_MAXP = 128;
constexpr int SW_PF = 12;

// Per-warp state with a buffer of BUF keys (8.6 KB for the 1,024 of
// select16_kernel, so that six CTAs of four warps fit on an SM).  The
// histogram is dead when the ties at the cut are collected, and the sample is
// dead when the compaction fills the buffer, so each pair shares its space.
template <int BUF>
struct SwStateT {
  static constexpr int kBuf = BUF;
  union {
    int hist[256];
    uint64_t ties[SW_TIE];  // (candidate position << 32 | index) of the keys at the cut
  } h;
  int sh[2], n, cnt, ecnt;
  int lid[SW_MAXP], nl[SW_MAXP], pst[SW_MAXP + 1];
  union {
    uint16_t samp[SW_SAMPLE];
    struct {
      uint16_t key[BUF];
      uint32_t idx[BUF];
    } b;
  } u;
};
using SwState = SwStateT<SW_BUF>;
// the survivors of the filtered scan: about kk from the nearest list plus those
// of the other lists under its bound, over 1,024 for a few percent of queries
constexpr int SV_BUF = 2048;

// the kth smallest (1-based, kth <= n) of n 16-bit keys, by one warp
template <class KeyF, class St>
__device__ __forceinline__ uint32_t warp_kth16(int n, int kth, KeyF key, St &s, int &below,
                                               int &neq) {
  return warp_radix_kth<2>(n, kth, key, s.h.hist, s.sh, below, neq);
}

// The kk smallest of n keys into o[0, kk) (any order): key(i), database
// entry id(i), candidate position pos(i).  kq > 0: winners above the kq-th
// smallest key + prune_delta become -1.  Keys equal to the cut are taken by
// ascending position: a warp sort of up to SW_TIE of them, else a prefix count
// (keys in position order) or a radix select on their positions.
// key_limit: every candidate key below it is among the n (the set may lack
// larger ones).  When the keys up to the pruning bound are all present and
// number at most kk, they are the winners that survive the pruning (they all
// rank within the kk smallest), so they are written directly, -1 after them,
// without the kk-th key or its ties.
template <bool ORDERED, class KeyF, class IdF, class PosF, class St>
__device__ __forceinline__ bool warp_select16(int n, int kk, int kq, int prune_delta, KeyF key, IdF id, PosF pos,
                              int64_t *o, St &s, uint32_t key_limit = 0) {
  const int lane = threadIdx.x & 31;
  uint32_t keep_max = 0xFFFFFFFFu;
  if (kq > 0) {
    int b2, n2;
    keep_max = warp_kth16(n, kq, key, s, b2, n2) + (uint32_t)prune_delta;
    // (a wide bound, as at FP8 precision, rarely leaves kk or fewer keys under
    // it: the count is not tried there)
    if (keep_max < key_limit && prune_delta <= 1024) {
      int c = 0;
      for (int i = lane; i < n; i += 32) c += key(i) <= keep_max ? 1 : 0;
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o2);
      if (c <= kk) {
        int base = 0;
        for (int i0 = 0; i0 < n; i0 += 32) {
          const int i = i0 + lane;
          const bool in = i < n && key(i) <= keep_max;
          const unsigned b = __ballot_sync(0xffffffffu, in);
          if (in) o[base + __popc(b & lanemask_lt())] = id(i);
          base += __popc(b);
        }
        for (int r = c + lane; r < kk; r += 32) o[r] = -1;
        __syncwarp();
        return true;
      }
    }
  }
  int below, neq;
  const uint32_t T = warp_kth16(n, kk, key, s, below, neq);
  if (lane == 0) s.cnt = s.ecnt = 0;
  __syncwarp();
  const int need_eq = kk - below;
  const bool few_ties = neq <= SW_TIE;
  for (int i = lane; i < n; i += 32) {
    const uint32_t k = key(i);
    if (k < T) {
      o[atomicAdd(&s.cnt, 1)] = k <= keep_max ? id(i) : -1;
    } else if (k == T && few_ties) {
      const int p = atomicAdd(&s.ecnt, 1);
      if (p < SW_TIE) s.h.ties[p] = ((uint64_t)(uint32_t)pos(i) << 32) | (uint32_t)i;
    }
  }
  __syncwarp();
  if (few_ties) {
    warp_sort(s.h.ties, neq);
    for (int j = lane; j < need_eq; j += 32)
      o[below + j] = T <= keep_max ? id((int)(uint32_t)(s.h.ties[j] & 0xffffffffu)) : -1;
  } else if (ORDERED) {
    // many ties, keys in position order: rank them with warp prefix counts
    int base = 0;
    for (int i0 = 0; i0 < n && base < need_eq; i0 += 32) {
      const int i = i0 + lane;
      const bool eq = i < n && key(i) == T;
      const unsigned b = __ballot_sync(0xffffffffu, eq);
      const int before = base + __popc(b & lanemask_lt());
      if (eq && before < need_eq) o[below + before] = T <= keep_max ? id(i) : -1;
      base += __popc(b);
    }
  } else {
    // many ties, keys not in position order: the need_eq-th smallest position
    // among them (positions are distinct) bounds the ones taken
    int b2, n2;
    const uint32_t posT = warp_radix_kth<4>(
        n, need_eq, [&](int i) -> uint32_t { return key(i) == T ? (uint32_t)pos(i) : 0xFFFFFFFFu; },
        s.h.hist, s.sh, b2, n2);
    if (lane == 0) s.ecnt = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32)
      if (key(i) == T && (uint32_t)pos(i) <= posT) {
        const int p = atomicAdd(&s.ecnt, 1);
        if (p < need_eq) o[below + p] = T <= keep_max ? id(i) : -1;
      }
  }
  __syncwarp();
  return true;
}

__global__ void __launch_bounds__(SW_WARPS * 32, 6) select16_kernel(
    const uint16_t *__restrict__ cand, const uint64_t *__restrict__ ckeys, int nprobe,
    const int64_t *__restrict__ qbase, const int64_t *__restrict__ list_off, int kk, int k,
    const float *__restrict__ qrho, float rmax, float e_rest, int prune, int64_t B,
    int64_t *__restrict__ out, unsigned long long *__restrict__ stats) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  SwState &s = ((SwState *)smem)[warp];
  const int64_t q = (int64_t)blockIdx.x * SW_WARPS + warp;
  if (q >= B) return;
  int prune_delta = 0;
  if (prune) {
    const double rq = (double)qrho[q];
    const double E = 2.0 * (rmax + rq + rmax * rq) * (1.0 + 1e-3) + e_rest;
    prune_delta = (int)ceil(2.0 * 16384.0 * (ldexp(1.0, -15) + E)) + 1;
    if (prune_delta > (1 << 20)) prune_delta = 1 << 20;
  }
  // probed lists: ids, sizes, padded starts (warp scan over 4 entries per lane)
  int ln[4], pl[4], tot = 0, ptot = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int sl = lane * 4 + j;
    ln[j] = 0;
    if (sl < nprobe) {
      const int l = probe_list(ckeys[q * nprobe + sl]);
      s.lid[sl] = l;
      ln[j] = l >= 0 ? (int)(list_off[l + 1] - list_off[l]) : 0;
      s.nl[sl] = ln[j];
    }
    pl[j] = (ln[j] + 7) & ~7;
    tot += ln[j];
    ptot += pl[j];
  }
  int inc = ptot;
#pragma unroll
  for (int o2 = 1; o2 < 32; o2 <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o2);
    if (lane >= o2) inc += y;
  }
  {
    int run = inc - ptot;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int sl = lane * 4 + j;
      if (sl <= nprobe) s.pst[sl] = run;
      run += pl[j];
    }
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o2);
  const int ptotal = __shfl_sync(0xffffffffu, inc, 31);
  const int total = tot;
  __syncwarp();
  int64_t *o = out + q * kk;
  auto id_at = [&](int i) -> int64_t {
    int lo = 0, hi = nprobe - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s.pst[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int m = i - s.pst[lo];
    return m < s.nl[lo] ? (((int64_t)s.lid[lo] << 32) | (int64_t)m) : -1;
  };
  if (total <= kk) {
    int p0 = 0;
    for (int sl = 0; sl < nprobe; ++sl) {
      const int nl = s.nl[sl];
      for (int m = lane; m < nl; m += 32) o[p0 + m] = ((int64_t)s.lid[sl] << 32) | (int64_t)m;
      p0 += nl;
    }
    for (int r = total + lane; r < kk; r += 32) o[r] = -1;
    return;
  }
  const int kq = prune ? k : 0;
  const uint16_t *src = cand + qbase[q];
  if (ptotal > 2 * SW_BUF) {
    // 1. threshold from a sample of evenly spaced runs of 8 keys
    const uint4 *g = (const uint4 *)src;
    const int nvec = ptotal >> 3;
    const int nrun = min(SW_SAMPLE / 8, nvec), ns = 8 * nrun;
    const uint64_t step = ((uint64_t)nvec << 20) / (uint64_t)nrun;  // 2^-20 units
    for (int j = lane; j < nrun; j += 32) {
      const uint4 v = g[(int)(((uint64_t)j * step) >> 20)];
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) s.u.samp[8 * j + e] = (uint16_t)((w[e >> 1] >> ((e & 1) * 16)) & 0xFFFFu);
    }
    __syncwarp();
    int r = (int)((0.5 * (kk + SW_BUF) * ns) / ptotal);
    r = max(0, min(r, ns - 1));
    int b_, n_;
    const uint32_t kv =
        warp_kth16(ns, r + 1, [&](int i) -> uint32_t { return s.u.samp[i]; }, s, b_, n_);
    if (kv < 0xFFFFu) {
      const uint32_t T = kv + 1;  // keys strictly below T survive
      if (lane == 0) s.n = 0;
      __syncwarp();
      // 2. compaction.  Two keys per 32-bit word are compared with T at once
      //    (SWAR: d = (x | H) - (T & ~H) cannot borrow across the halves; the
      //    half x < T iff (~x_top & T_top) | (~(x_top ^ T_top) & ~d_top)); the
      //    survivor flags go to bit 8e + 7 of a 64-bit mask for key e of the
      //    16-byte group; a lane with survivors claims its slots with one
      //    shared-memory atomic
      const uint32_t TT = T | (T << 16), TL = TT & 0x7FFF7FFFu;
      // two halves of SW_PF / 2 groups per lane: one half loads while the
      // other is compared
      constexpr int HB = SW_PF / 2;
      auto load = [&](uint4(&v)[HB], int cb) {
#pragma unroll
        for (int f = 0; f < HB; ++f) {
          const int c = cb + f * 32 + lane;
          v[f] = c < nvec ? g[c] : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        }
      };
      auto compact = [&](const uint4(&v)[HB], int cb) {
#pragma unroll
        for (int f = 0; f < HB; ++f) {
          const int c = cb + f * 32 + lane;
          const uint32_t w[4] = {v[f].x, v[f].y, v[f].z, v[f].w};
          uint32_t lt[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t x = w[i], d = (x | 0x80008000u) - TL;
            lt[i] = ((~x & TT) | (~(x ^ TT) & ~d)) & 0x80008000u;
          }
          uint64_t M = ((uint64_t)__byte_perm(lt[2], lt[3], 0x7531) << 32) |
                       (uint64_t)__byte_perm(lt[0], lt[1], 0x7531);
          if (M) {
            int p = atomicAdd(&s.n, __popcll(M));
            const uint64_t k01 = ((uint64_t)w[1] << 32) | w[0], k23 = ((uint64_t)w[3] << 32) | w[2];
            while (M) {
              const int e = (__ffsll((long long)M) - 1) >> 3;
              M &= M - 1;
              if (p < SW_BUF) {
                s.u.b.key[p] = (uint16_t)(((e < 4 ? k01 : k23) >> (16 * (e & 3))) & 0xFFFFu);
                s.u.b.idx[p] = (uint32_t)(c * 8 + e);
              }
              ++p;
            }
          }
        }
      };
      uint4 va[HB], vb[HB];
      load(va, 0);
      for (int c0 = 0; c0 < nvec; c0 += 2 * 32 * HB) {
        load(vb, c0 + 32 * HB);
        compact(va, c0);
        load(va, c0 + 2 * 32 * HB);
        compact(vb, c0 + 32 * HB);
      }
      __syncwarp();
      const int n = s.n;
      if (stats && lane == 0) atomicAdd(stats, (unsigned long long)n);
      // 3. exact select on the buffer
      if (n >= kk && n <= SW_BUF &&
          warp_select16<false>(n, kk, kq, prune_delta,
                               [&](int i) -> uint32_t { return s.u.b.key[i]; },
                               [&](int i) -> int64_t { return id_at((int)s.u.b.idx[i]); },
                               [&](int i) -> int { return (int)s.u.b.idx[i]; }, o, s, T))
        return;
    }
    if (stats && lane == 0) atomicAdd(stats + 1, 1ull);  // the buffer path failed
  }
  // exact select over the whole region (index = candidate position)
  warp_select16<true>(ptotal, kk, kq, prune_delta, [&](int i) -> uint32_t { return src[i]; }, id_at,
                      [&](int i) -> int { return i; }, o, s, 0x10000u);
}

// ---------------------------------------------------------------- filtered scan
// With the filtered tensor-core scan, each (query, probe slot) pair keeps only
// its members whose key can still be in the shortlist, as records
// (key << 16 | member index) compacted at the start of the pair's segment.
// A first pass scans every query's nearest list (slot 0) and writes all of its
// keys; their kk-th smallest, tau, bounds the query's overall kk-th key (those
// kk members are candidates too), so slot 0 keeps its records with key <= tau
// and the second pass over the other slots keeps keys <= tau only.  The
// shortlist is then selected from the survivors with the same (key, candidate
// position) order as select16_kernel, so the result is the same.

constexpr int TAU_WARPS = 4;

// Per query (one warp): tau = the kk-th smallest of slot 0's n0 keys (0xFFFF
// when n0 < kk) and slot 0's records with key <= tau, in member order.
__global__ void __launch_bounds__(TAU_WARPS * 32) shortlist_tau_kernel(
    const uint16_t *__restrict__ cand0, int64_t stride0, const uint64_t *__restrict__ ckeys,
    const int64_t *__restrict__ list_off, uint32_t *__restrict__ rec, int *__restrict__ rcnt,
    const int64_t *__restrict__ pbase, int nprobe, int kk, int64_t B,
    uint16_t *__restrict__ tau) {
  __shared__ int hist[TAU_WARPS][256];
  __shared__ int sh[TAU_WARPS][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * TAU_WARPS + warp;
  if (q >= B) return;
  const int64_t p0 = q * nprobe;
  const int l = probe_list(ckeys[p0]);  // slot 0 is never masked
  const int n0 = l >= 0 ? (int)(list_off[l + 1] - list_off[l]) : 0;
  const uint16_t *keys = cand0 + q * stride0;
  uint32_t T = 0xFFFFu;
  if (n0 >= kk) {
    int below, neq;
    T = warp_radix_kth<2>(n0, kk, [&](int i) -> uint32_t { return keys[i]; }, hist[warp],
                          sh[warp], below, neq);
  }
  uint32_t *r = rec + pbase[p0];
  int w = 0;
  for (int i0 = 0; i0 < n0; i0 += 32) {
    const int i = i0 + lane;
    const uint32_t k = i < n0 ? keys[i] : 0xFFFFFFFFu;
    const bool keep = i < n0 && k <= T;
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if (keep) r[w + __popc(b & lanemask_lt())] = (k << 16) | (uint32_t)i;
    w += __popc(b);
  }
  if (lane == 0) {
    rcnt[p0] = w;
    tau[q] = (uint16_t)T;
  }
}

struct SvState {
  SwStateT<SV_BUF> s;
  int spre[SW_MAXP + 1];  // survivors before each slot
  int64_t pb[SW_MAXP];    // record segment start of each slot
};

// Per query (one warp): the kk smallest (key, candidate position) among the
// survivors, written like select16_kernel (pruning included).
__global__ void __launch_bounds__(SW_WARPS * 32, 3) select_surv_kernel(
    const uint32_t *__restrict__ rec, const int *__restrict__ rcnt,
    const int64_t *__restrict__ pbase, const uint64_t *__restrict__ ckeys, int nprobe,
    const int64_t *__restrict__ list_off, int kk, int k, const float *__restrict__ qrho,
    float rmax, float e_rest, int prune, int64_t B, int64_t *__restrict__ out,
    unsigned long long *__restrict__ stats) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  SvState &v = ((SvState *)smem)[warp];
  auto &s = v.s;
  const int64_t q = (int64_t)blockIdx.x * SW_WARPS + warp;
  if (q >= B) return;
  int prune_delta = 0;
  if (prune) {
    const double rq = (double)qrho[q];
    const double E = 2.0 * (rmax + rq + rmax * rq) * (1.0 + 1e-3) + e_rest;
    prune_delta = (int)ceil(2.0 * 16384.0 * (ldexp(1.0, -15) + E)) + 1;
    if (prune_delta > (1 << 20)) prune_delta = 1 << 20;
  }
  // probed lists: ids, sizes, padded candidate starts, survivor counts
  int ln[4], pl[4], sc[4], tot = 0, ptot = 0, stot = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int sl = lane * 4 + j;
    ln[j] = 0;
    sc[j] = 0;
    if (sl < nprobe) {
      const int64_t p = q * nprobe + sl;
      const int l = probe_list(ckeys[p]);
      s.lid[sl] = l;
      ln[j] = l >= 0 ? (int)(list_off[l + 1] - list_off[l]) : 0;
      s.nl[sl] = ln[j];
      sc[j] = rcnt[p];
      v.pb[sl] = pbase[p];
    }
    pl[j] = (ln[j] + 7) & ~7;
    tot += ln[j];
    ptot += pl[j];
    stot += sc[j];
  }
  int inc = ptot, sinc = stot;
#pragma unroll
  for (int o2 = 1; o2 < 32; o2 <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o2);
    const int z = __shfl_up_sync(0xffffffffu, sinc, o2);
    if (lane >= o2) {
      inc += y;
      sinc += z;
    }
  }
  {
    int run = inc - ptot, srun = sinc - stot;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int sl = lane * 4 + j;
      if (sl <= nprobe) {
        s.pst[sl] = run;
        v.spre[sl] = srun;
      }
      run += pl[j];
      srun += sc[j];
    }
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o2);
  const int total = tot;
  const int S = __shfl_sync(0xffffffffu, sinc, 31);
  if (stats && lane == 0) {
    atomicAdd(stats, (unsigned long long)S);
    if (S > SV_BUF && total > kk) atomicAdd(stats + 1, 1ull);
  }
  __syncwarp();
  int64_t *o = out + q * kk;
  if (total <= kk) {
    int p0 = 0;
    for (int sl = 0; sl < nprobe; ++sl) {
      const int nl = s.nl[sl];
      for (int m = lane; m < nl; m += 32) o[p0 + m] = ((int64_t)s.lid[sl] << 32) | (int64_t)m;
      p0 += nl;
    }
    for (int r = total + lane; r < kk; r += 32) o[r] = -1;
    return;
  }
  // survivor i -> slot (last slot whose survivor prefix is <= i)
  auto slot_of = [&](int i) -> int {
    int lo = 0, hi = nprobe - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (v.spre[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  // candidate position -> (list << 32 | member)
  auto id_at = [&](int i) -> int64_t {
    int lo = 0, hi = nprobe - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s.pst[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int m = i - s.pst[lo];
    return m < s.nl[lo] ? (((int64_t)s.lid[lo] << 32) | (int64_t)m) : -1;
  };
  const int kq = prune ? k : 0;
  if (S <= SV_BUF) {
    for (int i = lane; i < S; i += 32) {
      const int sl = slot_of(i);
      const uint32_t r = rec[v.pb[sl] + (i - v.spre[sl])];
      s.u.b.key[i] = (uint16_t)(r >> 16);
      s.u.b.idx[i] = (uint32_t)(s.pst[sl] + (int)(r & 0xFFFFu));
    }
    __syncwarp();
    warp_select16<false>(S, kk, kq, prune_delta, [&](int i) -> uint32_t { return s.u.b.key[i]; },
                         [&](int i) -> int64_t { return id_at((int)s.u.b.idx[i]); },
                         [&](int i) -> int { return (int)s.u.b.idx[i]; }, o, s);
  } else {
    auto rec_at = [&](int i) -> uint32_t {
      const int sl = slot_of(i);
      return rec[v.pb[sl] + (i - v.spre[sl])];
    };
    auto pos_at = [&](int i) -> int {
      const int sl = slot_of(i);
      return s.pst[sl] + (int)(rec[v.pb[sl] + (i - v.spre[sl])] & 0xFFFFu);
    };
    warp_select16<false>(S, kk, kq, prune_delta, [&](int i) -> uint32_t { return rec_at(i) >> 16; },
                         [&](int i) -> int64_t { return id_at(pos_at(i)); }, pos_at, o, s);
  }
}

}  // namespace

int launch_shortlist_tau(const uint16_t *cand0, int64_t stride0, const uint64_t *ckeys,
                         const int64_t *list_off, uint32_t *rec, int *rcnt, const int64_t *pbase,
                         int nprobe, int kk, int64_t B, uint16_t *tau, cudaStream_t st) {
  if (B <= 0) return ADANNS_OK;
  shortlist_tau_kernel<<<(unsigned)((B + TAU_WARPS - 1) / TAU_WARPS), TAU_WARPS * 32, 0, st>>>(
      cand0, stride0, ckeys, list_off, rec, rcnt, pbase, nprobe, kk, B, tau);
  ADN_LAUNCH("shortlist_tau_kernel");
  return ADANNS_OK;
}

int launch_select_surv(const uint32_t *rec, const int *rcnt, const int64_t *pbase,
                       const uint64_t *ckeys, int nprobe, const int64_t *list_off, int kk, int k,
                       const float *qrho, float rmax, float e_rest, int prune, int64_t B,
                       int64_t *out, unsigned long long *stats, cudaStream_t st) {
  if (nprobe > SW_MAXP) return fail(ADANNS_ERR_ARG, "select: nprobe above 128");
  if (B <= 0) return ADANNS_OK;
  const size_t sm = sizeof(SvState) * SW_WARPS;
  ADN_CUDA(ensure_smem((const void *)select_surv_kernel, sm));
  select_surv_kernel<<<(unsigned)((B + SW_WARPS - 1) / SW_WARPS), SW_WARPS * 32, sm, st>>>(
      rec, rcnt, pbase, ckeys, nprobe, list_off, kk, k, qrho, rmax, e_rest, prune, B, out, stats);
  ADN_LAUNCH("select_surv_kernel");
  return ADANNS_OK;
}

int launch_select16(const uint16_t *cand, const uint64_t *ckeys, int nprobe, const int64_t *qbase,
                    const int64_t *list_off, int kk, int k, const float *qrho, float rmax,
                    float e_rest, int prune, int64_t B, int64_t *out, unsigned long long *stats,
                    cudaStream_t st) {
  if (nprobe > SW_MAXP) return fail(ADANNS_ERR_ARG, "select16: nprobe above 128");
  if (B <= 0) return ADANNS_OK;
  const size_t sm = sizeof(SwState) * SW_WARPS;
  ADN_CUDA(ensure_smem((const void *)select16_kernel, sm));
  select16_kernel<<<(unsigned)((B + SW_WARPS - 1) / SW_WARPS), SW_WARPS * 32, sm, st>>>(
      cand, ckeys, nprobe, qbase, list_off, kk, k, qrho, rmax, e_rest, prune, B, out, stats);
  ADN_LAUNCH("select16_kernel");
  return ADANNS_OK;
}

}  // namespace adn
