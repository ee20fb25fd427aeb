// Per-query selection of the kk smallest 32-bit keys over the query's
// candidate segments (the ADC distances of the probed lists, one FP32
// distance per member, whose bits order like the distances).  One CTA per
// query:
//  1. a sample of up to 8,192 keys (2,048 evenly spaced 16-byte runs) gives a
//     threshold T with about (kk + 4,096) / 2 smaller keys (radix select on
//     the sample);
//  2. one pass compacts every key < T, with its position, into a shared buffer;
//  3. if the buffer holds between kk and S32_BUF keys, an exact radix select
//     (four 8-bit digits) on the buffer fixes the cut, otherwise the same
//     select runs over the whole region.
// Ties at the cut go to the smallest database ids, so the kk keys are the kk
// smallest (distance, id) pairs, as a sort of the packed keys would give.
#include "devutil.cuh"
#include "internal.cuh"

namespace adn {
namespace {

constexpr int S32_THREADS = 256;
constexpr int S32_SAMPLE = 8192;  // keys sampled (2,048 runs of 4)
constexpr int S32_BUF = 4096;     // keys compacted below the threshold (same shared space)
constexpr int S32_TIE = 512;
constexpr int S32_UNROLL = 4;     // 16-byte loads in flight per thread in the compaction
constexpr int S32_MAXP = 256;  // probed lists per query

struct S32State {
  int hist[256];
  int sh[2], lt, eq;
  uint64_t ties[S32_TIE];  // (id << 32 | index) of the keys equal to the cut
};

// the kth smallest (1-based) of n keys; below = keys below it, neq = keys equal
template <class KeyF>
__device__ uint32_t radix_kth32(int n, int kth, KeyF key, S32State &st, int &below, int &neq) {
  return block_radix_kth<S32_THREADS, 4>(n, kth, key, st.hist, st.sh, &below, &neq);
}

// the kk smallest of n keys in (key, id) order: key(i), database id id(i)
// (distinct over the n keys, below 0xFFFFFFFF), output value val(i)
// (key << 32 | id), written to o[0, kk) in no particular order.  The keys equal
// to the cut go by ascending id: a warp sort when at most S32_TIE of them
// tie, else a second radix select on their ids.
template <class KeyF, class IdF, class ValF>
__device__ void select_into(int n, int kk, KeyF key, IdF id, ValF val, uint64_t *o, S32State &st) {
  const int tid = threadIdx.x;
  int below, neq;
  const uint32_t T = radix_kth32(n, kk, key, st, below, neq);
  const int need_eq = kk - below;
  if (tid == 0) st.lt = st.eq = 0;
  __syncthreads();
  for (int i = tid; i < n; i += S32_THREADS) {
    const uint32_t k = key(i);
    if (k < T) {
      o[atomicAdd(&st.lt, 1)] = val(i);
    } else if (k == T && neq <= S32_TIE) {
      const int p = atomicAdd(&st.eq, 1);
      if (p < S32_TIE) st.ties[p] = ((uint64_t)id(i) << 32) | (uint32_t)i;
    }
  }
  __syncthreads();
  if (neq <= S32_TIE) {
    if (tid < 32) {
      warp_sort(st.ties, neq);
      for (int j = tid; j < need_eq; j += 32) o[below + j] = val((int)(uint32_t)st.ties[j]);
    }
  } else {
    int b2, n2;
    const uint32_t idT = radix_kth32(
        n, need_eq, [&](int i) -> uint32_t { return key(i) == T ? id(i) : 0xFFFFFFFFu; }, st, b2,
        n2);
    if (tid == 0) st.eq = 0;
    __syncthreads();
    for (int i = tid; i < n; i += S32_THREADS)
      if (key(i) == T && id(i) <= idT) {
        const int p = atomicAdd(&st.eq, 1);
        if (p < need_eq) o[below + p] = val(i);
      }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(S32_THREADS) select32_kernel(
    const uint32_t *__restrict__ cand, const uint64_t *__restrict__ ckeys, int nprobe,
    const int64_t *__restrict__ qbase, const int64_t *__restrict__ list_off,
    const int32_t *__restrict__ list_ids, int kk, uint64_t *__restrict__ out) {
  __shared__ S32State st;
  // the sample, then (once the threshold is known) the compacted keys and positions
  __shared__ __align__(16) uint32_t space[S32_SAMPLE];
  uint32_t *samp = space, *bkey = space, *bidx = space + S32_BUF;
  __shared__ int s_n;
  __shared__ int64_t s_off[S32_MAXP];
  __shared__ int s_nl[S32_MAXP], s_pst[S32_MAXP + 1];
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int s = tid; s < nprobe; s += S32_THREADS) {
    const int l = probe_list(ckeys[q * nprobe + s]);
    s_off[s] = l >= 0 ? list_off[l] : 0;
    s_nl[s] = l >= 0 ? (int)(list_off[l + 1] - list_off[l]) : 0;
  }
  __syncthreads();
  if (tid == 0) {
    int t = 0;
    for (int s = 0; s < nprobe; ++s) { s_pst[s] = t; t += (s_nl[s] + 7) & ~7; }
    s_pst[nprobe] = t;
    s_n = 0;
  }
  __syncthreads();
  const int ptotal = s_pst[nprobe];
  int total = 0;
  for (int s = 0; s < nprobe; ++s) total += s_nl[s];
  uint64_t *o = out + q * kk;
  const uint32_t *src = cand + qbase[q];
  // value of candidate position i: (key << 32 | database id), KEY_MAX for padding
  auto val_at = [&](int i) -> uint64_t {
    int lo = 0, hi = nprobe - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pst[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int m = i - s_pst[lo];
    return m < s_nl[lo] ? (((uint64_t)src[i] << 32) | (uint32_t)list_ids[s_off[lo] + m]) : KEY_MAX;
  };
  auto id_at = [&](int i) -> uint32_t { return (uint32_t)(val_at(i) & 0xffffffffu); };
  if (total <= kk) {
    for (int s = 0; s < nprobe; ++s) {
      int p0 = 0;
      for (int s2 = 0; s2 < s; ++s2) p0 += s_nl[s2];
      for (int m = tid; m < s_nl[s]; m += S32_THREADS)
        o[p0 + m] = ((uint64_t)src[s_pst[s] + m] << 32) | (uint32_t)list_ids[s_off[s] + m];
    }
    for (int r = total + tid; r < kk; r += S32_THREADS) o[r] = KEY_MAX;
    return;
  }
  if (ptotal > 2 * S32_BUF) {
    // 1. threshold from a sample of up to S32_SAMPLE / 4 evenly spaced 16-byte
    //    runs, aimed at (kk + S32_BUF) / 2 keys below it
    const uint4 *g = (const uint4 *)src;
    const int nvec = ptotal >> 2;
    const int nrun = min(S32_SAMPLE / 4, nvec), ns = 4 * nrun;
    const uint64_t step = ((uint64_t)nvec << 20) / (uint64_t)nrun;  // 2^-20 units
    for (int j = tid; j < nrun; j += S32_THREADS) {
      const uint4 v = g[(int)(((uint64_t)j * step) >> 20)];
      samp[4 * j] = v.x;
      samp[4 * j + 1] = v.y;
      samp[4 * j + 2] = v.z;
      samp[4 * j + 3] = v.w;
    }
    __syncthreads();
    int r = (int)((0.5 * (kk + S32_BUF) * ns) / ptotal);
    r = max(0, min(r, ns - 1));
    int b2, n2;
    const uint32_t kv =
        radix_kth32(ns, r + 1, [&](int i) -> uint32_t { return samp[i]; }, st, b2, n2);
    __syncthreads();  // the sample's space is reused by the compaction
    if (kv != 0xFFFFFFFFu) {
      const uint32_t T = kv + 1;  // keys strictly below T survive
      // 2. compact the keys below T: S32_UNROLL 16-byte loads in flight per
      //    thread; a warp votes once per load and skips the word-by-word
      //    ranking when none of its 128 keys survives (the common case)
      for (int c0 = 0; c0 < nvec; c0 += S32_THREADS * S32_UNROLL) {
        uint4 v[S32_UNROLL];
#pragma unroll
        for (int u = 0; u < S32_UNROLL; ++u) {
          const int c = c0 + u * S32_THREADS + tid;
          v[u] = c < nvec ? g[c] : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        }
#pragma unroll
        for (int u = 0; u < S32_UNROLL; ++u) {
          const int c = c0 + u * S32_THREADS + tid;
          const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
          const uint32_t lo = min(min(w[0], w[1]), min(w[2], w[3]));
          if (!__any_sync(0xffffffffu, lo < T)) continue;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const bool take = w[e] < T;
            const unsigned m = __ballot_sync(0xffffffffu, take);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&s_n, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (take) {
              const int p = base + __popc(m & lanemask_lt());
              if (p < S32_BUF) {
                bkey[p] = w[e];
                bidx[p] = (uint32_t)(4 * c + e);
              }
            }
          }
        }
      }
      __syncthreads();
      const int n = s_n;
      if (n >= kk && n <= S32_BUF) {
        select_into(n, kk, [&](int i) -> uint32_t { return bkey[i]; },
                    [&](int i) -> uint32_t { return id_at((int)bidx[i]); },
                    [&](int i) -> uint64_t { return val_at((int)bidx[i]); }, o, st);
        return;
      }
    }
  }
  // 3. exact select over the whole region (index = candidate position)
  select_into(ptotal, kk, [&](int i) -> uint32_t { return src[i]; }, id_at,
              [&](int i) -> uint64_t { return val_at(i); }, o, st);
}

}  // namespace

namespace {
__global__ void keys_to_ids_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                   int64_t *__restrict__ ids) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ids[i] = keys[i] == KEY_MAX ? -1 : (int64_t)(uint32_t)(keys[i] & 0xffffffffu);
}
}  // namespace

int launch_keys_to_ids(const uint64_t *keys, int64_t n, int64_t *ids, cudaStream_t st) {
  if (n <= 0) return ADANNS_OK;
  keys_to_ids_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, n, ids);
  ADN_LAUNCH("keys_to_ids_kernel");
  return ADANNS_OK;
}

int launch_select32(const uint32_t *cand, const uint64_t *ckeys, int nprobe, const int64_t *qbase,
                    const int64_t *list_off, const int32_t *list_ids, int64_t B, int kk,
                    uint64_t *out, cudaStream_t st) {
  if (nprobe > S32_MAXP) return fail(ADANNS_ERR_ARG, "select32: nprobe above 256");
  if (B <= 0) return ADANNS_OK;
  select32_kernel<<<(unsigned)B, S32_THREADS, 0, st>>>(cand, ckeys, nprobe, qbase, list_off,
                                                       list_ids, kk, out);
  ADN_LAUNCH("select32_kernel");
  return ADANNS_OK;
}

}  // namespace adn
