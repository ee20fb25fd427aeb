// Mixed-precision AdANNS-IVF list scan on the 5th-generation tensor cores.
//
// The database is stored BF16 or FP8-E4M3 with a per-vector FP32 scale, in the
// same prefix-major list layout as the FP32 copy but with blocks of 128 bytes
// (64 BF16 or 128 FP8 coordinates).  For a work item (list, up to 128 queries
// probing it) the CTA computes the 128 x n_l matrix of dot products
//     D = Q_tile (128 x d_s) . X_list^T (d_s x n_l)
// with tcgen05.mma (FP32 accumulation in tensor memory), 256 members at a time,
// and turns each dot product into an approximate squared distance
//     d ~ |q|^2 + |x|^2 - 2 s_q s_x nu_x (q . x)
// (prefix-normalised metric, so d lies in [0, 4]), written as a 16-bit
// fixed-point key round(d * 2^14) into the query's candidate segment.  A selection kernel then keeps each query's best k' candidates and
// the exact FP32 rerank (Sec. 4.3 shortlist-rerank) produces the result.
//
// Warp roles (576 threads): warp 0 issues TMA tile loads into an NS-stage
// shared-memory ring (a stage is one K-block of 128 bytes per row of the query
// tile and of 256 members, 48 KB); warp 1 owns tensor memory (512 columns: two
// 256-column accumulators) and one elected thread issues the MMAs; warps 2-17
// drain the accumulators (four warps per TMEM lane quadrant, 64 columns each),
// staging SC key columns at a time in shared memory for row-segment stores.
// BF16 (a third of a microsecond of MMA work per stage) takes four stages, so
// that more loads are in flight, and 16-column staging to make room for them;
// FP8 (twice the MMA rate, the drain is the limit) keeps three stages and
// 64-column staging, whose stores are fewer and wider, except where few
// queries share a list (the loads are the limit there: four stages).  Every mbarrier wait is
// bounded: on timeout the kernel records an error, stops issuing work, lets
// in-flight copies land and frees TMEM.
#include <cuda.h>
#include <cuda_fp16.h>

#include <mutex>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {

namespace {
constexpr int BM = 128;          // queries per tile (TMEM lanes)
constexpr int BN = 256;          // members per MMA tile (TMEM columns per accumulator)
constexpr int ROWB = 128;        // bytes per K-block row (one 128-byte swizzle atom row)
constexpr int A_BYTES = BM * ROWB;    // 16 KB
constexpr int B_BYTES = BN * ROWB;    // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 16;                 // four per TMEM lane quadrant
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int EPI_SPAN = BN / (EPI_WARPS / 4);  // accumulator columns per epilogue warp
static_assert(EPI_SPAN == 64, "an epilogue warp drains 64 accumulator columns");
// a warp's key staging tile: 32 rows x SC keys (SC 16 or 64)
constexpr int stg_bytes(int sc) { return 32 * sc * 2; }
constexpr int THREADS = 64 + EPI_THREADS;
constexpr int TQD = 4;  // tile queue depth

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the phase with the given parity to complete (false once
// `limit_ns` of wall time has passed)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if ((i & 1023) == 1023) {
      const uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);           // start address
  d |= (uint64_t)0 << 16;                            // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;      // stride byte offset
  d |= (uint64_t)1 << 46;                            // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                            // layout: SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate, bool fp8) {
  if (fp8) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ int ld_abort(const int *flag) { return *(const volatile int *)flag; }

// bit e set for each of the 8 16-bit keys of v (key e in half e & 1 of word
// e >> 1) that is <= tau: two keys per word against T = tau + 1 (with
// d = (x | H) - (T & ~H) no borrow crosses the halves, and a half x < T iff
// (~x_top & T_top) | (~(x_top ^ T_top) & ~d_top))
__device__ __forceinline__ uint32_t keys_le8(const uint4 &v, uint32_t tau) {
  if (tau >= 0xFFFFu) return 0xFFu;
  const uint32_t T = tau + 1, TT = T | (T << 16), TL = TT & 0x7FFF7FFFu;
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t x = w[i], d = (x | 0x80008000u) - TL;
    const uint32_t lt = ((~x & TT) | (~(x ^ TT) & ~d)) & 0x80008000u;
    m |= ((lt >> 15) & 1u) << (2 * i) | (lt >> 31) << (2 * i + 1);
  }
  return m;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
}  // namespace



template <int NS, int SC>
__global__ void __launch_bounds__(THREADS, 1)
    mma_scan_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    MmaScanArgs a) {
  static_assert(SC == 16 || SC == 64, "staging of 16 or 64 key columns");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = smem;                          // NS x 16 KB
  unsigned char *sB = smem + NS * A_BYTES;           // NS x 32 KB
  unsigned char *sStage = smem + NS * STAGE_BYTES;   // EPI_WARPS x stg_bytes(SC) key staging
  __shared__ uint64_t full[NS], empty[NS], tfull[2], tempty[2], sfull[2];
  // tile queue: the producer takes tiles from a global counter (dynamic load
  // balance) and hands their ids to the MMA issuer and the epilogue in order
  __shared__ uint64_t qfull[TQD], qempty[TQD];
  __shared__ int qids[TQD];
  __shared__ __align__(16) float s_cb[2][BN];
  __shared__ __align__(16) float s_ca[2][BN];  // per member of the tile: -2 s_x nu_x, 2^14 |x|^2
  // filtered mode: survivors per tile row of the current and the previous work item
  __shared__ int s_rc[2][BM];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&tfull[s], 1);
      mbar_init(&tempty[s], EPI_THREADS);
      mbar_init(&sfull[s], EPI_THREADS);
    }
    for (int s = 0; s < TQD; ++s) {
      mbar_init(&qfull[s], 1);
      mbar_init(&qempty[s], 1 + EPI_THREADS);
    }
    abort_s = 0;
    for (int i = 0; i < 2 * BM; ++i) s_rc[i / BM][i % BM] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const int ntiles = *a.ntiles_dev;
  const uint32_t idesc = a.fp8 ? ((1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24))
                               : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                  ((uint32_t)(BM >> 4) << 24));

  // filtered mode: the last work item with member tiles whose survivor counts
  // this epilogue thread still has to write (see the epilogue)
  const bool filt = a.rec != nullptr && a.tau != nullptr;
  bool fl_pv = false;
  int fl_pp = 0, fl_buf = 0;
  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      int qs = 0;
      uint32_t qph = 0;
      for (;;) {
        int t = atomicAdd(a.tile_counter, 1);
        if (t >= ntiles || ld_abort(&abort_s)) t = -1;
        if (!mbar_wait(&qempty[qs], qph ^ 1, a.wait_ns)) {
          atomicExch(&abort_s, 1);
          atomicCAS(a.err, 0, 6);
          break;
        }
        qids[qs] = t;
        mbar_arrive(&qfull[qs]);
        if (++qs == TQD) { qs = 0; qph ^= 1; }
        if (t < 0) break;
        const int list = a.tile_list[t];
        const int64_t off = a.list_off[list];
        const int nl = (int)(a.list_off[list + 1] - off);
        const int nmt = (nl + BN - 1) / BN;
        for (int mt = 0; mt < nmt && !ld_abort(&abort_s); ++mt)
          for (int kb = 0; kb < a.nkb; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1, a.wait_ns)) {
              atomicExch(&abort_s, 1);
              atomicCAS(a.err, 0, 1);
              break;
            }
            // test hook: leave this stage of work item 0 unfilled (no copy, no
            // arrival), so the MMA issuer's bounded wait on it runs out
            if (t == 0 && mt * a.nkb + kb == a.skip_fill) {
              if (++stage == NS) { stage = 0; phase ^= 1; }
              continue;
            }
            mbar_expect_tx(&full[stage], STAGE_BYTES);
            tma_load_2d(sA + stage * A_BYTES, &tmA, &full[stage], 0, (t * a.nkb + kb) * BM);
            tma_load_2d(sB + stage * B_BYTES, &tmB, &full[stage], 0,
                        (int)(off * a.d_blocks) + kb * nl + mt * BN);
            if (++stage == NS) { stage = 0; phase ^= 1; }
          }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      int qs = 0;
      uint32_t qph = 0;
      while (!ld_abort(&abort_s)) {
        if (!mbar_wait(&qfull[qs], qph, a.wait_ns)) {
          atomicExch(&abort_s, 1);
          atomicCAS(a.err, 0, 7);
          break;
        }
        const int t = qids[qs];
        mbar_arrive(&qempty[qs]);
        if (++qs == TQD) { qs = 0; qph ^= 1; }
        if (t < 0) break;
        const int list = a.tile_list[t];
        const int nl = (int)(a.list_off[list + 1] - a.list_off[list]);
        const int nmt = (nl + BN - 1) / BN;
        for (int mt = 0; mt < nmt && !ld_abort(&abort_s); ++mt) {
          if (!mbar_wait(&tempty[acc], aphase ^ 1, a.wait_ns)) {
            atomicExch(&abort_s, 1);
            atomicCAS(a.err, 0, 2);
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
          for (int kb = 0; kb < a.nkb; ++kb) {
            if (!mbar_wait(&full[stage], phase, a.wait_ns)) {
              atomicExch(&abort_s, 1);
              atomicCAS(a.err, 0, 3);
              break;
            }
            tc_fence_after();
            const uint32_t abase = smem_u32(sA + stage * A_BYTES);
            const uint32_t bbase = smem_u32(sB + stage * B_BYTES);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              // 32 bytes of K per instruction: 16 BF16 or 32 FP8 elements
              mma_issue(d_tmem, sw128_desc(abase + ks * 32), sw128_desc(bbase + ks * 32), idesc,
                        (kb > 0 || ks > 0) ? 1u : 0u, a.fp8 != 0);
            }
            mma_commit(&empty[stage]);
            if (++stage == NS) { stage = 0; phase ^= 1; }
          }
          mma_commit(&tfull[acc]);
          if (++acc == 2) { acc = 0; aphase ^= 1; }
        }
      }
    }
  } else {
    // ---------------- epilogue: warps 2..17, one query row per thread; the
    // four warps of a TMEM lane quadrant (warp % 4) take a quarter of the
    // columns each
    const int quarter = warp & 3;
    const int c_lo = ((warp - 2) / 4) * EPI_SPAN;
    const int et = threadIdx.x - 64;
    const int row = quarter * 32 + lane;
    int acc = 0;
    uint32_t aphase = 0;
    int qs = 0;
    uint32_t qph = 0;
    // filtered mode: a pair's survivors are counted in s_rc[ib & 1][row] (shared
    // atomics of the row's four column warps) while its work item, the ib-th
    // with member tiles, is drained; at the next such item's first tile, after
    // the hand-off barrier that every epilogue thread passes only once done
    // with the previous tile, the first column warp of each quadrant writes
    // the count to rcnt and clears its slot for the item after that
    int ib = 0;
    for (;;) {
      if (!mbar_wait(&qfull[qs], qph, a.wait_ns)) {
        atomicExch(&abort_s, 1);
        atomicCAS(a.err, 0, 8);
        break;
      }
      const int t = qids[qs];
      mbar_arrive(&qempty[qs]);
      if (++qs == TQD) { qs = 0; qph ^= 1; }
      if (t < 0) break;
      const int list = a.tile_list[t];
      const int64_t off = a.list_off[list];
      const int nl = (int)(a.list_off[list + 1] - off);
      const int npad = (nl + 7) & ~7;
      const int nmt = (nl + BN - 1) / BN;
      const int cnt = a.tile_cnt[t];
      const bool valid = row < cnt;
      int64_t base = 0;
      float q2 = 0.f, qs = 0.f;
      uint32_t tau = 0xFFFFu;  // filtered mode: members with key <= tau survive
      int pidx = 0;
      if (valid) {
        const int p = a.pair_out[a.tile_beg[t] + row];
        const int q = p / a.nprobe;
        base = a.pstride ? (int64_t)(p / a.nprobe) * a.pstride : a.pbase[p];
        q2 = a.qn2[q];
        qs = a.qsc[q];
        pidx = p;
        if (a.tau) tau = a.tau[q];
      }
      const int cbuf = ib & 1;
      bool stop = false;
      // the row's terms in key units: key = round(clamp(d) * 2^14) with
      // d * 2^14 = (2^14 s_q) (-2 s_x nu_x) (q~ . x~) + 2^14 (|q|^2 + |x|^2);
      // scaling by 2^14 is exact, so the keys are those of the unscaled form
      const float qsk = 16384.f * qs, q2k = 16384.f * q2;
      // per-member terms of member tile mt (thread et < BN holds member et of
      // the tile), loaded one tile ahead so the loads overlap the drain
      auto load_terms = [&](int mt) -> float2 {
        float2 v = make_float2(0.f, 0.f);
        if (et < BN) {
          const int m = mt * BN + et;
          const float c = m < nl ? __ldg(a.cx + off + m) : 0.f;
          v.x = -2.f * c;
          // |x|^2 in key units (x 2^14, exact); members past the list end: huge
          v.y = m < nl ? 16384.f * (a.x2 ? __ldg(a.x2 + off + m) : (c > 0.f ? 1.f : 0.f)) : 3.0e38f;
        }
        return v;
      };
      float2 terms = load_terms(0);
      for (int mt = 0; mt < nmt; ++mt) {
        if (!mbar_wait(&tfull[acc], aphase, a.wait_ns)) {
          atomicExch(&abort_s, 1);
          atomicCAS(a.err, 0, 4);
          stop = true;
          break;
        }
        tc_fence_after();
        // the tile's per-member terms, staged once for the epilogue warps
        {
          if (et < BN) {
            s_cb[acc][et] = terms.x;
            s_ca[acc][et] = terms.y;
          }
          // hand-off through an mbarrier: a bounded wait, unlike bar.sync
          mbar_arrive(&sfull[acc]);
          if (!mbar_wait(&sfull[acc], aphase, a.wait_ns)) {
            atomicExch(&abort_s, 1);
            atomicCAS(a.err, 0, 5);
            stop = true;
            break;
          }
        }
        if (filt && mt == 0 && ib > 0 && c_lo == 0) {
          if (fl_pv) a.rcnt[fl_pp] = s_rc[fl_buf][row];
          s_rc[fl_buf][row] = 0;
        }
        if (mt + 1 < nmt) terms = load_terms(mt + 1);
        // a lane quadrant with no valid query row (a tile with few queries)
        // has nothing to drain: its warps skip the TMEM loads and the stores
        if (quarter * 32 < cnt) {
          const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN);
          // this warp's 32 rows of keys pass through a shared-memory tile of SC
          // columns (CPR 16-byte chunks per row, chunks XOR-swizzled by row so
          // that both the row-per-lane writes and the row-segment reads are
          // conflict-free) and are stored as SC * 2-byte row segments; in the
          // filtered pass a lane instead compares each 8-key chunk it reads
          // with its row's tau (two keys per word) and writes only the
          // survivors, as records, after one shared-memory atomic on the row's
          // count
          constexpr int CPR = SC / 8, LPR = CPR, RPI = 32 / LPR;
          uint4 *stg = (uint4 *)(sStage + (size_t)(warp - 2) * stg_bytes(SC));
          auto swz = [](int row, int ch) -> int {
            return CPR == 8 ? (ch ^ (row & 7)) : (ch ^ ((row >> 2) & 1));
          };
          const int chl = lane % LPR;
#pragma unroll 1
          for (int c0 = 0; c0 < EPI_SPAN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tbase + c_lo + c0, r);
            uint32_t packed[16];
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              // the four columns' member terms in one 16-byte read each
              const float4 cb = *(const float4 *)&s_cb[acc][c_lo + c0 + j];
              const float4 ca = *(const float4 *)&s_ca[acc][c_lo + c0 + j];
              const float cbv[4] = {cb.x, cb.y, cb.z, cb.w}, cav[4] = {ca.x, ca.y, ca.z, ca.w};
              uint32_t kk[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                // approximate squared distance as a 16-bit fixed-point key:
                // round(d * 2^14), d clamped to [0, 3.9999]; members past the
                // list end get the largest key.  The lower clamp is the
                // conversion's saturation.
                const float dk = fminf(fmaf(qsk * cbv[u], __uint_as_float(r[j + u]), q2k + cav[u]),
                                       3.9999f * 16384.f);
                asm("cvt.rni.sat.u32.f32 %0, %1;" : "=r"(kk[u]) : "f"(dk));
              }
              packed[j >> 1] = kk[0] | (kk[1] << 16);
              packed[(j >> 1) + 1] = kk[2] | (kk[3] << 16);
            }
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int col = c0 + 8 * g;  // column of this chunk in the warp's span
              stg[lane * CPR + swz(lane, (col % SC) / 8)] =
                  make_uint4(packed[4 * g], packed[4 * g + 1], packed[4 * g + 2], packed[4 * g + 3]);
              if ((col + 8) % SC == 0) {
                __syncwarp();
                // LPR lanes per row: one instruction stores RPI rows x SC * 2 bytes
                const int m0 = mt * BN + c_lo + col + 8 - SC;
#pragma unroll
                for (int i = 0; i < 32 / RPI; ++i) {
                  const int rr = i * RPI + lane / LPR;
                  const long long b = __shfl_sync(0xffffffffu, (long long)base, rr);
                  const int ok = __shfl_sync(0xffffffffu, valid ? 1 : 0, rr);
                  const uint32_t tr = __shfl_sync(0xffffffffu, tau, rr);
                  const uint4 v = stg[rr * CPR + swz(rr, chl)];
                  const int mb = m0 + 8 * chl;
                  if (!filt) {
                    if (ok && mb < npad) *(uint4 *)(a.cand + b + mb) = v;
                  } else if (ok && mb < nl) {
                    uint32_t msk = keys_le8(v, tr);
                    if (mb + 8 > nl) msk &= (1u << (nl - mb)) - 1u;  // members past the list end
                    if (msk) {
                      uint32_t *dst =
                          a.rec + b + atomicAdd(&s_rc[cbuf][quarter * 32 + rr], __popc(msk));
                      const uint64_t k01 = ((uint64_t)v.y << 32) | v.x,
                                     k23 = ((uint64_t)v.w << 32) | v.z;
                      while (msk) {
                        const int e = __ffs(msk) - 1;
                        msk &= msk - 1;
                        const uint32_t key =
                            (uint32_t)(((e < 4 ? k01 : k23) >> (16 * (e & 3))) & 0xFFFFu);
                        *dst++ = (key << 16) | (uint32_t)(mb + e);
                      }
                    }
                  }
                }
                __syncwarp();  // the staging tile is rewritten next
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[acc]);
        if (++acc == 2) { acc = 0; aphase ^= 1; }
      }
      if (stop) break;
      if (nmt > 0) {
        fl_pv = valid;
        fl_pp = pidx;
        fl_buf = cbuf;
        ++ib;
      }
      if (ld_abort(&abort_s)) break;
    }
  }

  __syncthreads();
  // filtered mode: the last work item's survivor counts (every epilogue thread
  // is past the block barrier, so they are final)
  if (filt && warp >= 2 && (warp - 2) / 4 == 0 && fl_pv && !ld_abort(&abort_s))
    a.rcnt[fl_pp] = s_rc[fl_buf][(warp & 3) * 32 + lane];
  if (ld_abort(&abort_s)) {
    // let any copy still in flight land before the shared memory is released
    for (int i = 0; i < 1 << 14; ++i) __nanosleep(1000);
  }
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------- narrow tiles
// The same scan for the memory-bound regime, where only a few queries probe
// each list.  The roles of the operands are swapped: a tile is 128 members
// (the MMA's M, TMEM lanes) by up to NQ = 32 queries (N, TMEM columns), so a
// pipeline stage holds 16 KB of member rows and 4 KB of query rows instead of
// 16 KB of mostly empty query rows and 32 KB of member rows: the stages in
// flight are nearly all database bytes, and the MMA no longer computes 128
// query rows for two or three live ones.  An epilogue thread holds one member
// and writes its keys for the tile's queries (a warp stores 32 consecutive
// members' keys per query).  The key arithmetic is the wide kernel's.
constexpr int NQ = 32;                      // queries per narrow tile (N)
constexpr int NMT = 128;                    // members per narrow tile (M)
constexpr int NA_BYTES = NMT * ROWB;        // 16 KB of member rows
constexpr int NB_BYTES = NQ * ROWB;         // 4 KB of query rows
constexpr int NACC = 4;                     // accumulators of NQ columns
constexpr int N_THREADS = 64 + 128;         // producer, MMA, four epilogue warps

template <int NS>
__global__ void __launch_bounds__(N_THREADS, 1)
    mma_narrow_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ,
                      MmaScanArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sX = smem;                    // NS x 16 KB member rows
  unsigned char *sQ = smem + NS * NA_BYTES;    // NS x 4 KB query rows
  __shared__ uint64_t full[NS], empty[NS], tfull[NACC], tempty[NACC];
  __shared__ uint64_t qfull[TQD], qempty[TQD];
  __shared__ int qids[TQD];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < NACC; ++s) {
      mbar_init(&tfull[s], 1);
      mbar_init(&tempty[s], 128);
    }
    for (int s = 0; s < TQD; ++s) {
      mbar_init(&qfull[s], 1);
      mbar_init(&qempty[s], 1 + 128);
    }
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(NACC * NQ));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const int ntiles = *a.ntiles_dev;
  const uint32_t idesc = a.fp8 ? ((1u << 4) | ((uint32_t)(NQ >> 3) << 17) | ((uint32_t)(NMT >> 4) << 24))
                               : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NQ >> 3) << 17) |
                                  ((uint32_t)(NMT >> 4) << 24));
  auto give_up = [&](int code) {
    atomicExch(&abort_s, 1);
    atomicCAS(a.err, 0, code);
  };
  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmX) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmQ) : "memory");
      int stage = 0, qs = 0;
      uint32_t phase = 0, qph = 0;
      for (;;) {
        int t = atomicAdd(a.tile_counter, 1);
        if (t >= ntiles || ld_abort(&abort_s)) t = -1;
        if (!mbar_wait(&qempty[qs], qph ^ 1, a.wait_ns)) {
          give_up(9);
          break;
        }
        qids[qs] = t;
        mbar_arrive(&qfull[qs]);
        if (++qs == TQD) { qs = 0; qph ^= 1; }
        if (t < 0) break;
        const int list = a.tile_list[t];
        const int64_t off = a.list_off[list];
        const int nl = (int)(a.list_off[list + 1] - off);
        const int nmt = (nl + NMT - 1) / NMT;
        bool ok = true;
        for (int mt = 0; mt < nmt && ok && !ld_abort(&abort_s); ++mt)
          for (int kb = 0; kb < a.nkb; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1, a.wait_ns)) {
              give_up(10);
              ok = false;
              break;
            }
            mbar_expect_tx(&full[stage], NA_BYTES + NB_BYTES);
            tma_load_2d(sX + stage * NA_BYTES, &tmX, &full[stage], 0,
                        (int)(off * a.d_blocks) + kb * nl + mt * NMT);
            tma_load_2d(sQ + stage * NB_BYTES, &tmQ, &full[stage], 0, (t * a.nkb + kb) * NQ);
            if (++stage == NS) { stage = 0; phase ^= 1; }
          }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: D[member][query] = X . Q^T
    if (lane == 0) {
      int stage = 0, acc = 0, qs = 0;
      uint32_t phase = 0, aphase = 0, qph = 0;
      while (!ld_abort(&abort_s)) {
        if (!mbar_wait(&qfull[qs], qph, a.wait_ns)) {
          give_up(11);
          break;
        }
        const int t = qids[qs];
        mbar_arrive(&qempty[qs]);
        if (++qs == TQD) { qs = 0; qph ^= 1; }
        if (t < 0) break;
        const int list = a.tile_list[t];
        const int nl = (int)(a.list_off[list + 1] - a.list_off[list]);
        const int nmt = (nl + NMT - 1) / NMT;
        bool ok = true;
        for (int mt = 0; mt < nmt && ok && !ld_abort(&abort_s); ++mt) {
          if (!mbar_wait(&tempty[acc], aphase ^ 1, a.wait_ns)) {
            give_up(12);
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem + (uint32_t)(acc * NQ);
          for (int kb = 0; kb < a.nkb; ++kb) {
            if (!mbar_wait(&full[stage], phase, a.wait_ns)) {
              give_up(13);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t xbase = smem_u32(sX + stage * NA_BYTES);
            const uint32_t qbase = smem_u32(sQ + stage * NB_BYTES);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_issue(d_tmem, sw128_desc(xbase + ks * 32), sw128_desc(qbase + ks * 32), idesc,
                        (kb > 0 || ks > 0) ? 1u : 0u, a.fp8 != 0);
            mma_commit(&empty[stage]);
            if (++stage == NS) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&tfull[acc]);
          if (++acc == NACC) { acc = 0; aphase ^= 1; }
        }
      }
    }
  } else {
    // ---------------- epilogue: warps 2..5, one member per thread (TMEM lane
    // quadrant warp % 4), the tile's queries as columns
    const int quarter = warp & 3;
    int acc = 0, qs = 0;
    uint32_t aphase = 0, qph = 0;
    for (;;) {
      if (!mbar_wait(&qfull[qs], qph, a.wait_ns)) {
        give_up(14);
        break;
      }
      const int t = qids[qs];
      mbar_arrive(&qempty[qs]);
      if (++qs == TQD) { qs = 0; qph ^= 1; }
      if (t < 0) break;
      const int list = a.tile_list[t];
      const int64_t off = a.list_off[list];
      const int nl = (int)(a.list_off[list + 1] - off);
      const int npad = (nl + 7) & ~7;
      const int nmt = (nl + NMT - 1) / NMT;
      const int cnt = a.tile_cnt[t];
      // lane j holds query column j's segment start and terms in key units
      long long base = 0;
      float qsk = 0.f, q2k = 0.f;
      if (lane < cnt) {
        const int p = a.pair_out[a.tile_beg[t] + lane];
        const int q = p / a.nprobe;
        base = a.pbase[p];
        qsk = 16384.f * a.qsc[q];
        q2k = 16384.f * a.qn2[q];
      }
      bool stop = false;
      for (int mt = 0; mt < nmt; ++mt) {
        const int m = mt * NMT + quarter * 32 + lane;
        float cb = 0.f, cak = 3.0e38f;  // members past the list end: the largest key
        if (m < nl) {
          const float c = __ldg(a.cx + off + m);
          cb = -2.f * c;
          cak = 16384.f * (a.x2 ? __ldg(a.x2 + off + m) : (c > 0.f ? 1.f : 0.f));
        }
        if (!mbar_wait(&tfull[acc], aphase, a.wait_ns)) {
          give_up(15);
          stop = true;
          break;
        }
        tc_fence_after();
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * NQ), r);
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
          if (j >= cnt) break;  // uniform in the warp
          const float qj = __shfl_sync(0xffffffffu, qsk, j);
          const float q2j = __shfl_sync(0xffffffffu, q2k, j);
          const long long bj = __shfl_sync(0xffffffffu, base, j);
          if (m < npad) {
            const float dk =
                fminf(fmaf(qj * cb, __uint_as_float(r[j]), q2j + cak), 3.9999f * 16384.f);
            uint32_t key;
            asm("cvt.rni.sat.u32.f32 %0, %1;" : "=r"(key) : "f"(dk));
            a.cand[bj + m] = (uint16_t)key;
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[acc]);
        if (++acc == NACC) { acc = 0; aphase ^= 1; }
      }
      if (stop || ld_abort(&abort_s)) break;
    }
  }
  __syncthreads();
  if (ld_abort(&abort_s)) {
    // let any copy still in flight land before the shared memory is released
    for (int i = 0; i < 1 << 14; ++i) __nanosleep(1000);
  }
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(NACC * NQ));
  }
}

// ---------------------------------------------------------------- host side
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// 2D map over rows of 128 bytes: box = 128 bytes x box_rows, 128-byte swizzle
int make_map(CUtensorMap *m, const void *base, int64_t rows, int box_rows, bool fp8) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(ADANNS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if (((uintptr_t)base & 15) != 0) return fail(ADANNS_ERR_ARG, "tensor base not 16-byte aligned");
  const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[2] = {(cuuint64_t)(fp8 ? 128 : 64), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {(cuuint32_t)(fp8 ? 128 : 64), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(ADANNS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return ADANNS_OK;
}
}  // namespace

static_assert(NQ == MMA_NARROW_QT, "narrow tile width shared with the host");
constexpr int NS_NARROW = 8;  // 8 x 20 KB stages

int launch_mma_narrow(const void *qtiles, int64_t qrows, const void *xlow, int64_t xrows,
                      const MmaScanArgs &a, cudaStream_t st) {
  if (a.rec || a.tau || a.pstride) return fail(ADANNS_ERR_ARG, "narrow scan: unfiltered keys only");
  CUtensorMap tX, tQ;
  int rc;
  if ((rc = make_map(&tX, xlow, xrows, NMT, a.fp8 != 0))) return rc;
  if ((rc = make_map(&tQ, qtiles, qrows, NQ, a.fp8 != 0))) return rc;
  MmaScanArgs b = a;
  b.wait_ns = (uint64_t)option(ADANNS_OPT_WAIT_LIMIT_NS);
  b.skip_fill = -1;
  const size_t smem = (size_t)NS_NARROW * (NA_BYTES + NB_BYTES) + 1024;
  ADN_CUDA(ensure_smem((const void *)mma_narrow_kernel<NS_NARROW>, smem));
  mma_narrow_kernel<NS_NARROW><<<num_sms(), N_THREADS, smem, st>>>(tX, tQ, b);
  ADN_LAUNCH("mma_narrow_kernel");
  return ADANNS_OK;
}

// stage count and staging width per element type (see the kernel's notes)
constexpr int NS_BF16 = 4, SC_BF16 = 16, NS_FP8 = 3, SC_FP8 = 64;
size_t mma_scan_smem(int ns, int sc) {
  return (size_t)ns * STAGE_BYTES + (size_t)EPI_WARPS * stg_bytes(sc) + 1024;
}

int launch_mma_scan(const void *qtiles, int64_t qrows, const void *xlow, int64_t xrows,
                    const MmaScanArgs &a, cudaStream_t st) {
  CUtensorMap tA, tB;
  int rc;
  if ((rc = make_map(&tA, qtiles, qrows, BM, a.fp8 != 0))) return rc;
  if ((rc = make_map(&tB, xlow, xrows, BN, a.fp8 != 0))) return rc;
  MmaScanArgs b = a;
  b.wait_ns = (uint64_t)option(ADANNS_OPT_WAIT_LIMIT_NS);
  b.skip_fill = (int)take_option(ADANNS_OPT_TEST_SKIP_LOAD, -1);
  if (a.fp8 && !a.few) {
    const size_t smem = mma_scan_smem(NS_FP8, SC_FP8);
    ADN_CUDA(ensure_smem((const void *)mma_scan_kernel<NS_FP8, SC_FP8>, smem));
    mma_scan_kernel<NS_FP8, SC_FP8><<<num_sms(), THREADS, smem, st>>>(tA, tB, b);
  } else {
    const size_t smem = mma_scan_smem(NS_BF16, SC_BF16);
    ADN_CUDA(ensure_smem((const void *)mma_scan_kernel<NS_BF16, SC_BF16>, smem));
    mma_scan_kernel<NS_BF16, SC_BF16><<<num_sms(), THREADS, smem, st>>>(tA, tB, b);
  }
  ADN_LAUNCH("mma_scan_kernel");
  return ADANNS_OK;
}

}  // namespace adn
