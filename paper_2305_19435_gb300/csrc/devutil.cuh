// Device helpers: async copies, warp sorting of packed (distance, id) keys.
#pragma once
#include <stdint.h>

namespace adn {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// L2 eviction-priority policies (per-access hints; no device state changes)
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async16_hint(void *smem, const void *gmem, uint64_t pol) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ float4 ldg_f4_hint(const float4 *p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// One full warp: the smallest bucket b of a 256-bucket histogram h with
// base + h[0] + ... + h[b] >= target, and the count below it
// (base + h[0] + ... + h[b-1]).  Needs target <= base + sum(h).
__device__ __forceinline__ void warp_find_bucket(const int *h, int base, int target, int *b_out,
                                                 int *below_out) {
  const int lane = threadIdx.x & 31;
  int v[8], sum = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v[j] = h[lane * 8 + j];
    sum += v[j];
  }
  int inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const unsigned m = __ballot_sync(0xffffffffu, base + inc >= target);
  const int L = m ? __ffs(m) - 1 : 31;
  if (lane == L) {
    // first bucket j of the lane's 8 whose running count reaches target
    int c = base + inc - sum, jb = 7;
    bool found = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!found) {
        if (j == 7 || c + v[j] >= target) {
          jb = j;
          found = true;
        } else {
          c += v[j];
        }
      }
    }
    *b_out = L * 8 + jb;
    *below_out = c;
  }
}

// One warp: the kth smallest (1-based, 1 <= kth <= n) of n keys key(i) of
// NPASS * 8 bits, by NPASS passes of 8-bit digits over the warp's 256-int
// shared histogram hist (sh: 2 shared ints).  below = keys smaller than the
// result, neq = keys equal to it.
template <int NPASS, class KeyF>
__device__ __forceinline__ uint32_t warp_radix_kth(int n, int kth, KeyF key, int *hist, int *sh,
                                                   int &below, int &neq) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0, mask = 0;
  int bl = 0;
#pragma unroll 1
  for (int pass = 0; pass < NPASS; ++pass) {
    const int shift = 8 * (NPASS - 1 - pass);
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const uint32_t k = key(i);
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1);
    }
    __syncwarp();
    warp_find_bucket(hist, bl, kth, sh, sh + 1);
    __syncwarp();
    const int digit = sh[0];
    prefix |= (uint32_t)digit << shift;
    mask |= 255u << shift;
    bl = sh[1];
    if (pass == NPASS - 1) neq = hist[digit];
    __syncwarp();
  }
  below = bl;
  return prefix;
}

// Block-wide radix select over n keys key(i) of NPASS * 8 bits: the kth
// smallest (1-based, 1 <= kth <= n) by NPASS passes of 8-bit digits, most
// significant first, over the 256-int shared histogram hist.  *below = keys
// smaller than the result, *neq = keys equal to it.  All NT threads of the
// block call it; sh is 2 shared ints; it ends with the block synchronised.
template <int NT, int NPASS, class KeyF>
__device__ uint32_t block_radix_kth(int n, int kth, KeyF key, int *hist, int *sh, int *below_out,
                                    int *neq_out) {
  const int tid = threadIdx.x;
  uint32_t prefix = 0, mask = 0;
  int below = 0, neq = 0;
  for (int pass = 0; pass < NPASS; ++pass) {
    const int shift = 8 * (NPASS - 1 - pass);
    for (int i = tid; i < 256; i += NT) hist[i] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
      const uint32_t k = key(i);
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1);
    }
    __syncthreads();
    if (tid < 32) warp_find_bucket(hist, below, kth, sh, sh + 1);
    __syncthreads();
    const int digit = sh[0];
    prefix |= (uint32_t)digit << shift;
    mask |= 255u << shift;
    below = sh[1];
    if (pass == NPASS - 1) neq = hist[digit];
    __syncthreads();  // hist and sh are rewritten by the next pass or the caller
  }
  *below_out = below;
  *neq_out = neq;
  return prefix;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

// Ascending sort of a[0:n) in shared memory by one warp.  Bitonic network in
// its "flip" form over the next power of two P >= n: every compare-exchange
// puts the smaller key at the lower index, so the missing elements [n, P)
// behave as +inf and are simply skipped.
__device__ __forceinline__ void warp_sort(uint64_t *a, int n) {
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < n) P <<= 1;
  const int pairs = P >> 1;
  for (int size = 2; size <= P; size <<= 1) {
    const int half = size >> 1;
    const int lh = __ffs(half) - 1;
    for (int p = lane; p < pairs; p += 32) {
      const int blk = p >> lh, off = p & (half - 1);
      const int i = blk * size + off, j = blk * size + size - 1 - off;
      if (j < n) {
        uint64_t x = a[i], y = a[j];
        if (y < x) { a[i] = y; a[j] = x; }
      }
    }
    __syncwarp();
    for (int stride = half >> 1; stride > 0; stride >>= 1) {
      const int ls = __ffs(stride) - 1;
      for (int p = lane; p < pairs; p += 32) {
        const int i = ((p >> ls) << (ls + 1)) + (p & (stride - 1)), j = i + stride;
        if (j < n) {
          uint64_t x = a[i], y = a[j];
          if (y < x) { a[i] = y; a[j] = x; }
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace adn
