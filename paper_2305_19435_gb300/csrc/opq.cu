// AdANNS-OPQ on the d_s prefix and the AdANNS-IVFOPQ search (Sec. 3 "OPQ",
// Sec. 4.2, Sec. 4.3, Table "formula" IVFOPQ row, read as asymmetric lookup):
//   * PQ: z = P_ds(x) R is split into M sub-vectors of d_s / M coordinates,
//     each quantised to the nearest of 256 codewords (one byte per subspace);
//   * OPQ training alternates Lloyd steps on the codebooks with the
//     orthogonal Procrustes rotation R = polar(Y^T Zhat);
//   * search: per query LUT[m][c] = ||z_m - C_m[c]||^2, and a member's
//     distance is the sum of its M table entries (M lookups per distance);
//   * optional exact rerank of the ADC shortlist with the FP32 d_s prefix.
#include <algorithm>
#include <vector>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {

// ---------------------------------------------------------------- PQ assignment
// grid (point blocks of 256, M); the subspace's codebook and the block's
// sub-vectors are staged in shared memory; ties go to the smallest codeword.
__global__ void pq_assign_kernel(const float *__restrict__ z, int64_t n, int ldz, int M,
                                 int dsub, const float *__restrict__ C,
                                 uint8_t *__restrict__ codes, float *__restrict__ mind) {
  extern __shared__ float ps[];
  float *Cs = ps;                  // [256][dsub]
  float *Zs = ps + 256 * dsub;     // [dsub][256]
  const int m = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const float *Cm = C + (int64_t)m * 256 * dsub;
  for (int e = threadIdx.x; e < 256 * dsub; e += 256) Cs[e] = Cm[e];
  if (i < n)
    for (int t = 0; t < dsub; ++t) Zs[t * 256 + threadIdx.x] = z[i * ldz + (int64_t)m * dsub + t];
  __syncthreads();
  if (i >= n) return;
  float best = __int_as_float(0x7f800000);
  int bc = 0;
  for (int c = 0; c < 256; ++c) {
    float acc = 0.f;
    for (int t = 0; t < dsub; ++t) {
      const float df = Zs[t * 256 + threadIdx.x] - Cs[c * dsub + t];
      acc = fmaf(df, df, acc);
    }
    if (acc < best) { best = acc; bc = c; }
  }
  codes[i * M + m] = (uint8_t)bc;
  if (mind) mind[i * M + m] = best;
}

int launch_pq_assign(const float *z, int64_t n, int ldz, int M, int dsub, const float *C,
                     uint8_t *codes, float *mind, cudaStream_t st) {
  if (n <= 0) return ADANNS_OK;
  const size_t smem = (size_t)512 * dsub * 4;
  ADN_CUDA(ensure_smem((const void *)pq_assign_kernel, (size_t)(smem)));
  dim3 grid((unsigned)((n + 255) / 256), M);
  pq_assign_kernel<<<grid, 256, smem, st>>>(z, n, ldz, M, dsub, C, codes, mind);
  ADN_LAUNCH("pq_assign_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- PQ update
__global__ void pq_accum_kernel(const float *__restrict__ z, int64_t n, int ldz, int M, int dsub,
                                const uint8_t *__restrict__ codes, double *__restrict__ sums,
                                int32_t *__restrict__ counts) {
  const int ds = M * dsub;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ds) return;
  const int64_t i = e / ds;
  const int j = (int)(e - i * ds);
  const int m = j / dsub, t = j - m * dsub;
  const int c = codes[i * M + m];
  atomicAdd(&sums[((int64_t)m * 256 + c) * dsub + t], (double)z[i * ldz + j]);
  if (t == 0) atomicAdd(&counts[m * 256 + c], 1);
}

__global__ void pq_finish_kernel(const double *__restrict__ sums,
                                 const int32_t *__restrict__ counts, int M, int dsub,
                                 float *__restrict__ C) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * 256 * dsub) return;
  const int mc = (int)(e / dsub);
  const int cnt = counts[mc];
  if (cnt > 0) C[e] = (float)(sums[e] / (double)cnt);
}

int launch_pq_update(const float *z, int64_t n, int ldz, int M, int dsub, const uint8_t *codes,
                     double *sums, int32_t *counts, float *C, cudaStream_t st) {
  const int64_t ne = (int64_t)M * 256 * dsub;
  ADN_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * ne, st));
  ADN_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * M * 256, st));
  const int64_t tot = n * M * dsub;
  if (tot > 0) {
    pq_accum_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(z, n, ldz, M, dsub, codes,
                                                                   sums, counts);
    ADN_LAUNCH("pq_accum_kernel");
  }
  pq_finish_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(sums, counts, M, dsub, C);
  ADN_LAUNCH("pq_finish_kernel");
  return ADANNS_OK;
}

__global__ void pq_decode_kernel(const uint8_t *__restrict__ codes, int64_t n, int M, int dsub,
                                 const float *__restrict__ C, float *__restrict__ out, int ldo) {
  const int ds = M * dsub;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ds) return;
  const int64_t i = e / ds;
  const int j = (int)(e - i * ds);
  const int m = j / dsub, t = j - m * dsub;
  out[i * ldo + j] = C[((int64_t)m * 256 + codes[i * M + m]) * dsub + t];
}

// sum of mind (per point per subspace) in FP64
__global__ void sum_f32_kernel(const float *__restrict__ v, int64_t n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (double)v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// ---------------------------------------------------------------- query LUT
// lut[q][m][c] = sum_t (z[q][m*dsub + t] - C[m][c][t])^2; grid (B, M), c = thread.
__global__ void pq_lut_kernel(const float *__restrict__ z, int ldz, int M, int dsub,
                              const float *__restrict__ C, float *__restrict__ lut) {
  const int64_t q = blockIdx.x;
  const int m = blockIdx.y, c = threadIdx.x;
  extern __shared__ float zq[];
  for (int t = threadIdx.x; t < dsub; t += 256) zq[t] = z[q * ldz + (int64_t)m * dsub + t];
  __syncthreads();
  const float *cw = C + ((int64_t)m * 256 + c) * dsub;
  float acc = 0.f;
  for (int t = 0; t < dsub; ++t) {
    const float df = zq[t] - cw[t];
    acc = fmaf(df, df, acc);
  }
  lut[(q * M + m) * 256 + c] = acc;
}

// ---------------------------------------------------------------- ADC list scan
struct AdcArgs {
  const uint8_t *codes;     // [N][M] in list order
  const int64_t *list_off;
  const int32_t *list_ids;
  int M;
  const float *lut;         // [B][M][256]
  const int32_t *tile_list, *tile_beg, *tile_cnt;
  const int *ntiles_dev;
  int *counter;
  const int32_t *pair_q, *pair_out;
  int k;
  uint64_t *out_keys;
};

constexpr int ADC_THREADS = 256;
constexpr int ADC_NW = ADC_THREADS / 32;
constexpr int ADC_MAXM = 64;  // code bytes held in registers by the fast path

// Work item = (list, up to QA queries that probe it).  The queries' LUTs sit in
// shared memory; each thread takes one member per chunk of 256, reads its M
// code bytes once and forms the M-lookup sum for every query of the tile;
// candidates beating the query's k-th key enter its buffer, which one warp per
// query sorts and trims after each chunk.
__global__ void __launch_bounds__(ADC_THREADS) adc_scan_kernel(AdcArgs a, int qa_max, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = a.M;
  const int lut_sz = M * 256;
  float *s_lut = (float *)smem;
  uint64_t *s_buf = (uint64_t *)(smem + (size_t)qa_max * lut_sz * 4);
  uint64_t *s_scr = s_buf + (size_t)qa_max * cap;
  uint64_t *s_tau = s_scr + (size_t)qa_max * cap;
  int *s_cnt = (int *)(s_tau + qa_max);
  int *s_na = s_cnt + qa_max;
  int *s_qrow = s_na + qa_max;
  int *s_orow = s_qrow + qa_max;
  __shared__ int s_tile;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = *a.ntiles_dev;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    const int list = a.tile_list[tile], beg = a.tile_beg[tile], cnt = a.tile_cnt[tile];
    if (tid < qa_max) {
      const bool v = tid < cnt;
      s_qrow[tid] = v ? a.pair_q[beg + tid] : -1;
      s_orow[tid] = v ? a.pair_out[beg + tid] : -1;
      s_cnt[tid] = 0;
      s_na[tid] = 0;
      s_tau[tid] = KEY_MAX;
    }
    __syncthreads();
    for (int e = tid; e < cnt * (lut_sz / 4); e += ADC_THREADS) {
      const int qa = e / (lut_sz / 4), r = e - qa * (lut_sz / 4);
      ((float4 *)s_lut)[(size_t)qa * (lut_sz / 4) + r] =
          ((const float4 *)(a.lut + (int64_t)s_qrow[qa] * lut_sz))[r];
    }
    __syncthreads();
    const int64_t off = a.list_off[list];
    const int nl = (int)(a.list_off[list + 1] - off);
    const int nchunk = (nl + ADC_THREADS - 1) / ADC_THREADS;
    for (int c = 0; c < nchunk; ++c) {
      const int mem = c * ADC_THREADS + tid;
      if (mem < nl) {
        const uint32_t id = (uint32_t)a.list_ids[off + mem];
        const uint8_t *cp = a.codes + (off + mem) * (int64_t)M;
        auto offer = [&](int qa, float d) {
          const uint64_t key = pack_key(d, id);
          if (key < s_tau[qa]) {
            const int pos = atomicAdd(&s_cnt[qa], 1);
            s_buf[(size_t)qa * cap + pos] = key;
          }
        };
        if ((M & 3) == 0 && M <= ADC_MAXM) {
          // the member's code words stay in registers; four queries at a time,
          // each with four partial sums (one per byte of a word), so sixteen
          // independent lookup chains are in flight
          uint32_t cw[ADC_MAXM / 4];
#pragma unroll
          for (int w = 0; w < ADC_MAXM / 4; ++w)
            if (w < (M >> 2)) cw[w] = ((const uint32_t *)cp)[w];
          for (int qa0 = 0; qa0 < cnt; qa0 += 4) {
            float sum[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
              for (int b = 0; b < 4; ++b) sum[j][b] = 0.f;
#pragma unroll
            for (int w = 0; w < ADC_MAXM / 4; ++w) {
              if (w >= (M >> 2)) break;
              const uint32_t word = cw[w];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (qa0 + j >= cnt) break;
                const float *Lw = s_lut + (size_t)(qa0 + j) * lut_sz + w * 4 * 256;
                sum[j][0] += Lw[word & 0xff];
                sum[j][1] += Lw[256 + ((word >> 8) & 0xff)];
                sum[j][2] += Lw[512 + ((word >> 16) & 0xff)];
                sum[j][3] += Lw[768 + (word >> 24)];
              }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (qa0 + j < cnt) offer(qa0 + j, (sum[j][0] + sum[j][1]) + (sum[j][2] + sum[j][3]));
          }
        } else {
          for (int qa = 0; qa < cnt; ++qa) {
            const float *L = s_lut + (size_t)qa * lut_sz;
            float d = 0.f;
            for (int m = 0; m < M; ++m) d += L[m * 256 + cp[m]];
            offer(qa, d);
          }
        }
      }
      __syncthreads();
      const bool last = c == nchunk - 1;
      for (int qa = warp; qa < cnt; qa += ADC_NW) {
        const int n = s_cnt[qa], na = s_na[qa];
        if (n > cap - ADC_THREADS || (last && n > na)) {
          uint64_t *buf = s_buf + (size_t)qa * cap;
          uint64_t *scr = s_scr + (size_t)qa * cap;
          // sort the new keys, merge with the sorted prefix, keep k
          warp_sort(buf + na, n - na);
          const int keep = n < a.k ? n : a.k;
          const int nb = n - na;
          for (int i = lane; i < na && i < keep; i += 32) {
            int lo = 0, hi = nb;
            const uint64_t key = buf[i];
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (buf[na + mid] < key) lo = mid + 1; else hi = mid; }
            if (i + lo < keep) scr[i + lo] = key;
          }
          for (int j = lane; j < nb && j < keep; j += 32) {
            int lo = 0, hi = na;
            const uint64_t key = buf[na + j];
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (buf[mid] < key) lo = mid + 1; else hi = mid; }
            if (j + lo < keep) scr[j + lo] = key;
          }
          __syncwarp();
          for (int i = lane; i < keep; i += 32) buf[i] = scr[i];
          __syncwarp();
          if (lane == 0) {
            s_cnt[qa] = keep;
            s_na[qa] = keep;
            s_tau[qa] = keep == a.k ? buf[a.k - 1] : KEY_MAX;
          }
        }
      }
      __syncthreads();
    }
    for (int qa = warp; qa < cnt; qa += ADC_NW) {
      uint64_t *out = a.out_keys + (int64_t)s_orow[qa] * a.k;
      const int n = s_cnt[qa];
      const uint64_t *buf = s_buf + (size_t)qa * cap;
      for (int r = lane; r < a.k; r += 32) out[r] = r < n ? buf[r] : KEY_MAX;
    }
    __syncthreads();
  }
}

static int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// queries per ADC work item: their LUTs (M KB each) plus two top-k buffers
// of next_pow2(k) + 256 keys must fit in about 200 KB of shared memory
int adc_query_tile(int M, int k) {
  const int cap = next_pow2(k) + ADC_THREADS;
  const int per_q = M * 256 * 4 + 2 * cap * 8 + 24;
  const int qa = (200 * 1024) / per_q;
  return std::max(1, std::min(8, qa));
}

int launch_adc_scan(const AdcArgs &a, int qa, cudaStream_t st) {
  const int cap = next_pow2(a.k) + ADC_THREADS;
  const size_t smem = (size_t)qa * a.M * 256 * 4 + (size_t)2 * qa * cap * 8 + (size_t)qa * 8 +
                      (size_t)qa * 16;
  if (smem > 220 * 1024) return fail(ADANNS_ERR_ARG, "ADC tile does not fit in shared memory");
  ADN_CUDA(ensure_smem((const void *)adc_scan_kernel, (size_t)(smem)));
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adc_scan_kernel, ADC_THREADS, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  adc_scan_kernel<<<num_sms() * per_sm, ADC_THREADS, smem, st>>>(a, qa, cap);
  ADN_LAUNCH("adc_scan_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- exact rerank
// One warp per query: the kr candidate ids are re-scored with the exact FP32
// difference-form distance on the d_s prefix (read from the prefix-major
// storage, 8 lanes per candidate), then the k best by (distance, id) are kept.
constexpr int RR_WARPS = 4;

__global__ void rerank_kernel(const int64_t *__restrict__ cand, int kr, int64_t B,
                              const float *__restrict__ qs, int ldq, int d_s,
                              const float *__restrict__ xpm, int d_pad,
                              const int64_t *__restrict__ list_off,
                              const int32_t *__restrict__ assign, const int32_t *__restrict__ pos,
                              const float *__restrict__ mscale, int k, int cap,
                              int64_t *__restrict__ out_ids, float *__restrict__ out_dist) {
  extern __shared__ __align__(16) unsigned char rsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * RR_WARPS + warp;
  float *sq = (float *)rsm + (size_t)warp * ldq;
  uint64_t *buf = (uint64_t *)((float *)rsm + (size_t)RR_WARPS * ldq) + (size_t)warp * cap;
  if (q >= B) return;
  for (int j = lane; j < ldq; j += 32) sq[j] = qs[q * ldq + j];
  __syncwarp();
  const int g = lane >> 3, s = lane & 7;
  const int nseg = d_s >> 2;  // float4 segments (d_s is a multiple of 8)
  for (int r0 = 0; r0 < kr; r0 += 4) {
    const int r = r0 + g;
    const int64_t id = r < kr ? cand[q * kr + r] : -1;
    float acc = 0.f;
    if (id >= 0) {
      const int l = assign[id];
      const int64_t p = pos[id];
      const int64_t off = list_off[l];
      const int64_t nl = list_off[l + 1] - off;
      const float *base = xpm + off * d_pad + (p - off) * 16;
      const float nu = mscale ? mscale[p] : 1.f;
      for (int e = s; e < nseg; e += 8) {
        const int b = e >> 2, part = e & 3;
        const float4 x = *(const float4 *)(base + (int64_t)b * 16 * nl + part * 4);
        const float4 qv = *(const float4 *)(sq + e * 4);
        float t;
        t = fmaf(-nu, x.x, qv.x); acc = fmaf(t, t, acc);
        t = fmaf(-nu, x.y, qv.y); acc = fmaf(t, t, acc);
        t = fmaf(-nu, x.z, qv.z); acc = fmaf(t, t, acc);
        t = fmaf(-nu, x.w, qv.w); acc = fmaf(t, t, acc);
      }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    if (s == 0 && r < kr) buf[r] = id >= 0 ? pack_key(acc, (uint32_t)id) : KEY_MAX;
  }
  __syncwarp();
  warp_sort(buf, kr);
  for (int r = lane; r < k; r += 32) {
    const uint64_t key = r < kr ? buf[r] : KEY_MAX;
    out_ids[q * k + r] = key == KEY_MAX ? -1 : (int64_t)(uint32_t)(key & 0xffffffffu);
    out_dist[q * k + r] = key == KEY_MAX ? __int_as_float(0x7f800000)
                                         : __uint_as_float((uint32_t)(key >> 32));
  }
}

int launch_rerank(const int64_t *cand, int kr, int64_t B, const float *qs, int ldq, int d_s,
                  const adanns_index *idx, const float *mscale, int k, int64_t *out_ids,
                  float *out_dist, cudaStream_t st) {
  if (B <= 0) return ADANNS_OK;
  const int cap = kr;
  const size_t smem = (size_t)RR_WARPS * ldq * 4 + (size_t)RR_WARPS * cap * 8;
  ADN_CUDA(ensure_smem((const void *)rerank_kernel, (size_t)(smem)));
  rerank_kernel<<<(unsigned)((B + RR_WARPS - 1) / RR_WARPS), RR_WARPS * 32, smem, st>>>(
      cand, kr, B, qs, ldq, d_s, idx->xpm, idx->d_pad, idx->list_off, idx->assign, idx->pos_of_id,
      mscale, k, cap, out_ids, out_dist);
  ADN_LAUNCH("rerank_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- misc
__global__ void permute_codes_kernel(const uint8_t *__restrict__ by_id,
                                     const int32_t *__restrict__ list_ids, int64_t N, int M,
                                     uint8_t *__restrict__ lo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * M) return;
  const int64_t p = e / M;
  const int m = (int)(e - p * M);
  lo[e] = by_id[(int64_t)list_ids[p] * M + m];
}

__global__ void identity_kernel(float *R, int d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  R[e] = (e / d) == (e % d) ? 1.f : 0.f;
}

__global__ void frob_kernel(const float *__restrict__ A, int64_t n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (double)A[i] * (double)A[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// X <- a * X + b * Y (elementwise), and ||X^T X - I||_F^2 pieces
__global__ void axpby_kernel(float *X, const float *Y, int64_t n, float a, float b) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) X[e] = a * X[e] + b * Y[e];
}

__global__ void orth_err_kernel(const float *__restrict__ G, int d, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)G[e] - ((e / d) == (e % d) ? 1.0 : 0.0);
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

int launch_gemm_f32(bool transA, int M, int N, int K, float alpha, const float *A, int lda,
                    const float *B, int ldb, float beta, float *C, int ldc, cudaStream_t st);

// Orthogonal polar factor of the d x d matrix Mx (= U V^T for Mx = U S V^T,
// the Procrustes solution of min ||Y R - Zhat|| over orthogonal R when
// Mx = Y^T Zhat): Newton-Schulz iteration X <- 1.5 X - 0.5 X (X^T X) from
// X0 = Mx / ||Mx||_F, until ||X^T X - I||_F < 1e-6 (at most 200 steps).
int polar_factor(const float *Mx, int d, float *R, cudaStream_t st) {
  Scratch s(st);
  float *X, *G, *T;
  double *acc;
  int rc;
  const int64_t dd = (int64_t)d * d;
  if ((rc = s.get(&X, dd)) || (rc = s.get(&G, dd)) || (rc = s.get(&T, dd)) || (rc = s.get(&acc, 1)))
    return rc;
  ADN_CUDA(cudaMemsetAsync(acc, 0, sizeof(double), st));
  frob_kernel<<<64, 256, 0, st>>>(Mx, dd, acc);
  ADN_LAUNCH("frob_kernel");
  double nrm2 = 0.0;
  ADN_CUDA(cudaMemcpyAsync(&nrm2, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  ADN_CUDA(cudaStreamSynchronize(st));
  if (!(nrm2 > 0.0)) return fail(ADANNS_ERR_ARG, "Procrustes matrix is zero");
  ADN_CUDA(cudaMemcpyAsync(X, Mx, sizeof(float) * dd, cudaMemcpyDeviceToDevice, st));
  const unsigned g = (unsigned)((dd + 255) / 256);
  axpby_kernel<<<g, 256, 0, st>>>(X, X, dd, (float)(1.0 / sqrt(nrm2)), 0.f);
  ADN_LAUNCH("axpby_kernel");
  for (int it = 0; it < 200; ++it) {
    if ((rc = launch_gemm_f32(true, d, d, d, 1.f, X, d, X, d, 0.f, G, d, st))) return rc;
    if (it % 4 == 3) {
      ADN_CUDA(cudaMemsetAsync(acc, 0, sizeof(double), st));
      orth_err_kernel<<<64, 256, 0, st>>>(G, d, acc);
      ADN_LAUNCH("orth_err_kernel");
      double err = 0.0;
      ADN_CUDA(cudaMemcpyAsync(&err, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
      ADN_CUDA(cudaStreamSynchronize(st));
      if (sqrt(err) < 1e-6) break;
    }
    if ((rc = launch_gemm_f32(false, d, d, d, 1.f, X, d, G, d, 0.f, T, d, st))) return rc;
    axpby_kernel<<<g, 256, 0, st>>>(X, T, dd, 1.5f, -0.5f);
    ADN_LAUNCH("axpby_kernel");
  }
  ADN_CUDA(cudaMemcpyAsync(R, X, sizeof(float) * dd, cudaMemcpyDeviceToDevice, st));
  return ADANNS_OK;
}

int launch_pq_lut(const float *z, int64_t B, int ldz, int M, int dsub, const float *C, float *lut,
                  cudaStream_t st) {
  if (B <= 0) return ADANNS_OK;
  dim3 grid((unsigned)B, M);
  pq_lut_kernel<<<grid, 256, dsub * 4, st>>>(z, ldz, M, dsub, C, lut);
  ADN_LAUNCH("pq_lut_kernel");
  return ADANNS_OK;
}

int launch_pq_decode(const uint8_t *codes, int64_t n, int M, int dsub, const float *C, float *out,
                     int ldo, cudaStream_t st) {
  const int64_t tot = n * M * dsub;
  if (tot <= 0) return ADANNS_OK;
  pq_decode_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(codes, n, M, dsub, C, out, ldo);
  ADN_LAUNCH("pq_decode_kernel");
  return ADANNS_OK;
}

int launch_sum_f32(const float *v, int64_t n, double *out, cudaStream_t st) {
  ADN_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  if (n <= 0) return ADANNS_OK;
  sum_f32_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4 * num_sms()), 256, 0, st>>>(
      v, n, out);
  ADN_LAUNCH("sum_f32_kernel");
  return ADANNS_OK;
}

int launch_sum_sq(const float *v, int64_t n, double *out, cudaStream_t st) {
  ADN_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  if (n <= 0) return ADANNS_OK;
  frob_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4 * num_sms()), 256, 0, st>>>(v, n,
                                                                                             out);
  ADN_LAUNCH("frob_kernel");
  return ADANNS_OK;
}

int launch_adc(const uint8_t *codes, const int64_t *list_off, const int32_t *list_ids, int M,
               const float *lut, const int32_t *tl, const int32_t *tb, const int32_t *tc,
               const int *ntiles, int *counter, const int32_t *pair_q, const int32_t *pair_out,
               int k, uint64_t *out_keys, int qa, cudaStream_t st) {
  AdcArgs a{};
  a.codes = codes;
  a.list_off = list_off;
  a.list_ids = list_ids;
  a.M = M;
  a.lut = lut;
  a.tile_list = tl;
  a.tile_beg = tb;
  a.tile_cnt = tc;
  a.ntiles_dev = ntiles;
  a.counter = counter;
  a.pair_q = pair_q;
  a.pair_out = pair_out;
  a.k = k;
  a.out_keys = out_keys;
  return launch_adc_scan(a, qa, st);
}

int launch_permute_codes(const uint8_t *by_id, const int32_t *list_ids, int64_t N, int M,
                         uint8_t *lo, cudaStream_t st) {
  const int64_t tot = N * M;
  if (tot <= 0) return ADANNS_OK;
  permute_codes_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(by_id, list_ids, N, M, lo);
  ADN_LAUNCH("permute_codes_kernel");
  return ADANNS_OK;
}

int launch_identity(float *R, int d, cudaStream_t st) {
  identity_kernel<<<(unsigned)(((int64_t)d * d + 255) / 256), 256, 0, st>>>(R, d);
  ADN_LAUNCH("identity_kernel");
  return ADANNS_OK;
}


// ---------------------------------------------------------------- ADC distances
// Distances first, selection after (adanns_search_ivfopq for nprobe <= 256):
// a work item = (list, up to QA queries probing it) computes the exact FP32
// ADC distance of every member for each query (the same four partial sums
// per code word as adc_scan_kernel) and writes its bits into the pair's
// candidate segment (the segment's padding to 8 gets 0xFFFFFFFF).  No
// per-query state is kept, so QA is bounded by the lookup tables alone.
struct AdcDistArgs {
  const uint8_t *codes;     // [N][M] in list order
  const int64_t *list_off;
  int M;
  const float *lut;         // [B][M][256]
  const int32_t *tile_list, *tile_beg, *tile_cnt;
  const int *ntiles_dev;
  int *counter;
  const int32_t *pair_q, *pair_out;
  const int64_t *pbase;     // candidate segment start of each pair
  uint32_t *cand;           // FP32 distance bits
  int nsplit;               // member ranges per tile (work items = tiles x nsplit)
  // residual codes (res_S NULL: plain): per-list tables S [nlist][M][256],
  // list centres rotated w [nlist][d_s] and |w|^2, queries rotated z [B][d_s]
  const float *res_S, *res_w, *res_w2, *z;
  int d_s;
};

constexpr int AD_THREADS = 256;
constexpr int AD_MAXQA = 16;

template <int G> struct LutVec;
template <> struct LutVec<4> { using T = float4; };
template <> struct LutVec<2> { using T = float2; };
template <> struct LutVec<1> { using T = float; };
__device__ __forceinline__ float lane_of(const float4 &v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
__device__ __forceinline__ float lane_of(const float2 &v, int j) { return j == 0 ? v.x : v.y; }
__device__ __forceinline__ float lane_of(const float &v, int) { return v; }

// Work item = (list, up to qa queries).  The tile's tables are staged
// query-interleaved in groups of G queries, [group][m][code][G], so one
// shared-memory load of G floats serves G queries' lookups of one code byte.
// One thread per member: its code words stay in registers; per query four
// partial sums (byte b of each word into sum[b]), combined as
// (s0 + s1) + (s2 + s3), the same arithmetic as the running top-k scan.
// Every probed member's distance bits go to the query's candidate segment,
// padding slots [n_l, pad8(n_l)) get 0xFFFFFFFF.
template <int G>
__global__ void __launch_bounds__(AD_THREADS) adc_dist_kernel(AdcDistArgs a) {
  using V = typename LutVec<G>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = a.M;
  const int lut_sz = M * 256;
  float *s_lut = (float *)smem;
  const V *s_lv = (const V *)smem;
  __shared__ int s_qrow[AD_MAXQA];
  __shared__ int64_t s_pb[AD_MAXQA];
  __shared__ float s_K[AD_MAXQA];  // residual codes: w2_l - 2 <w_l, z_q> per query of the tile
  __shared__ int s_tile;
  const int tid = threadIdx.x;
  const int nitems = *a.ntiles_dev * a.nsplit;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_tile;
    if (item >= nitems) break;
    const int tile = item / a.nsplit, range = item - tile * a.nsplit;
    const int list = a.tile_list[tile], beg = a.tile_beg[tile], cnt = a.tile_cnt[tile];
    const int ng = (cnt + G - 1) / G;
    if (tid < cnt) {
      s_qrow[tid] = a.pair_q[beg + tid];
      s_pb[tid] = a.pbase[a.pair_out[beg + tid]];
    }
    __syncthreads();
    // residual codes: this list's table is added to every query's table, and
    // the per-query constant |w_l|^2 - 2 <w_l, z_q> goes to the score
    const float *Sl = a.res_S ? a.res_S + (int64_t)list * lut_sz : nullptr;
    if (a.res_S) {
      const int warp = tid >> 5, lane = tid & 31;
      const float *wl = a.res_w + (int64_t)list * a.d_s;
      for (int j = warp; j < cnt; j += AD_THREADS / 32) {
        const float *zq = a.z + (int64_t)s_qrow[j] * a.d_s;
        float dot = 0.f;
        for (int t = lane; t < a.d_s; t += 32) dot = fmaf(wl[t], zq[t], dot);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) s_K[j] = fmaf(-2.f, dot, a.res_w2[list]);
      }
    }
    for (int g = 0; g < ng; ++g) {
      const float *src[G];
#pragma unroll
      for (int j = 0; j < G; ++j)
        src[j] = g * G + j < cnt ? a.lut + (int64_t)s_qrow[g * G + j] * lut_sz : nullptr;
      V *dst = (V *)s_lut + (size_t)g * lut_sz;
      for (int r = tid; r < lut_sz; r += AD_THREADS) {
        union {
          V v;
          float f[G];
        } u;
        const float sl = Sl ? Sl[r] : 0.f;
#pragma unroll
        for (int j = 0; j < G; ++j) u.f[j] = src[j] ? src[j][r] + sl : 0.f;
        dst[r] = u.v;
      }
    }
    __syncthreads();
    const int64_t off = a.list_off[list];
    const int nl = (int)(a.list_off[list + 1] - off);
    const int npad = (nl + 7) & ~7;
    // this item's chunks of AD_THREADS members: range `range` of nsplit
    const int nch = (npad + AD_THREADS - 1) / AD_THREADS;
    const int cper = (nch + a.nsplit - 1) / a.nsplit;
    const int m_end = min(npad, min(nch, (range + 1) * cper) * AD_THREADS);
    for (int m0 = range * cper * AD_THREADS; m0 < m_end; m0 += AD_THREADS) {
      const int mem = m0 + tid;
      if (mem < nl) {
        const uint8_t *cp = a.codes + (off + mem) * (int64_t)M;
        if ((M & 3) == 0 && M <= ADC_MAXM) {
          uint32_t cw[ADC_MAXM / 4];
#pragma unroll
          for (int w = 0; w < ADC_MAXM / 4; ++w)
            if (w < (M >> 2)) cw[w] = ((const uint32_t *)cp)[w];
          for (int g = 0; g < ng; ++g) {
            const V *Lg = s_lv + (size_t)g * lut_sz;
            float sum[G][4];
#pragma unroll
            for (int j = 0; j < G; ++j)
#pragma unroll
              for (int b = 0; b < 4; ++b) sum[j][b] = 0.f;
#pragma unroll
            for (int w = 0; w < ADC_MAXM / 4; ++w) {
              if (w >= (M >> 2)) break;
              const uint32_t word = cw[w];
              const V *Lw = Lg + w * 4 * 256;
              const V v0 = Lw[word & 0xff], v1 = Lw[256 + ((word >> 8) & 0xff)],
                      v2 = Lw[512 + ((word >> 16) & 0xff)], v3 = Lw[768 + (word >> 24)];
#pragma unroll
              for (int j = 0; j < G; ++j) {
                sum[j][0] += lane_of(v0, j);
                sum[j][1] += lane_of(v1, j);
                sum[j][2] += lane_of(v2, j);
                sum[j][3] += lane_of(v3, j);
              }
            }
#pragma unroll
            for (int j = 0; j < G; ++j)
              if (g * G + j < cnt) {
                float d = (sum[j][0] + sum[j][1]) + (sum[j][2] + sum[j][3]);
                if (Sl) d = fmaxf(d + s_K[g * G + j], 0.f);
                a.cand[s_pb[g * G + j] + mem] = __float_as_uint(d);
              }
          }
        } else {
          for (int qa = 0; qa < cnt; ++qa) {
            const float *L = s_lut + (size_t)(qa / G) * lut_sz * G + (qa % G);
            float d = 0.f;
            for (int m = 0; m < M; ++m) d += L[(m * 256 + cp[m]) * G];
            if (Sl) d = fmaxf(d + s_K[qa], 0.f);
            a.cand[s_pb[qa] + mem] = __float_as_uint(d);
          }
        }
      } else if (mem < npad) {
        for (int qa = 0; qa < cnt; ++qa) a.cand[s_pb[qa] + mem] = 0xFFFFFFFFu;
      }
    }
    __syncthreads();  // the next tile's tables overwrite these
  }
}

// queries interleaved per table entry: 4 when a group of 4 tables fits in
// ~200 KB of shared memory, else 2, else 1
int adc_dist_group(int M) {
  const int t = M * 256 * 4;
  return 4 * t <= 200 * 1024 ? 4 : 2 * t <= 200 * 1024 ? 2 : 1;
}

// queries per ADC distance work item: whole groups of tables within ~200 KB
int adc_dist_query_tile(int M) {
  const int G = adc_dist_group(M), t = M * 256 * 4;
  return std::max(1, std::min(AD_MAXQA, (200 * 1024) / (G * t) * G));
}

int launch_adc_dist(const uint8_t *codes, const int64_t *list_off, int M, const float *lut,
                    const int32_t *tl, const int32_t *tb, const int32_t *tc, const int *ntiles,
                    int *counter, const int32_t *pair_q, const int32_t *pair_out,
                    const int64_t *pbase, uint32_t *cand, int qa, int nsplit, cudaStream_t st,
                    const float *res_S, const float *res_w, const float *res_w2, const float *z,
                    int d_s) {
  AdcDistArgs a{};
  a.res_S = res_S;
  a.res_w = res_w;
  a.res_w2 = res_w2;
  a.z = z;
  a.d_s = d_s;
  a.nsplit = nsplit < 1 ? 1 : nsplit;
  a.codes = codes;
  a.list_off = list_off;
  a.M = M;
  a.lut = lut;
  a.tile_list = tl;
  a.tile_beg = tb;
  a.tile_cnt = tc;
  a.ntiles_dev = ntiles;
  a.counter = counter;
  a.pair_q = pair_q;
  a.pair_out = pair_out;
  a.pbase = pbase;
  a.cand = cand;
  const int G = adc_dist_group(M);
  const size_t smem = (size_t)((qa + G - 1) / G) * G * M * 256 * 4;
  const void *fn = G == 4 ? (const void *)adc_dist_kernel<4>
                   : G == 2 ? (const void *)adc_dist_kernel<2>
                            : (const void *)adc_dist_kernel<1>;
  ADN_CUDA(ensure_smem(fn, smem));
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, AD_THREADS, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  void *args[] = {&a};
  ADN_CUDA(cudaLaunchKernel(fn, dim3(num_sms() * per_sm), dim3(AD_THREADS), args, smem, st));
  ADN_LAUNCH("adc_dist_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- residual codes
// lcent[l] = mean over the members of list l of their d_s prefixes (times the
// inverse prefix norm under the prefix-normalised metric), FP64 sums; one CTA
// per list, one thread per coordinate (strided).  Empty lists get zeros.
__global__ void list_mean_kernel(const float *__restrict__ xpm, int d_pad,
                                 const int64_t *__restrict__ list_off,
                                 const float *__restrict__ mscale, int d_s,
                                 float *__restrict__ lcent) {
  const int l = blockIdx.x;
  const int64_t off = list_off[l];
  const int64_t nl = list_off[l + 1] - off;
  const float *base = xpm + off * d_pad;
  for (int j = threadIdx.x; j < d_s; j += blockDim.x) {
    double acc = 0.0;
    const float *col = base + (int64_t)(j >> 4) * 16 * nl + (j & 15);
    for (int64_t m = 0; m < nl; ++m)
      acc += (double)col[m * 16] * (double)(mscale ? mscale[off + m] : 1.f);
    lcent[(int64_t)l * d_s + j] = nl > 0 ? (float)(acc / (double)nl) : 0.f;
  }
}

int launch_list_mean(const adanns_index *x, int d_s, float *lcent, cudaStream_t st) {
  const float *mscale = x->metric == ADANNS_METRIC_L2_PREFIXNORM
                            ? x->invn + (int64_t)gran_index(d_s) * x->N
                            : nullptr;
  list_mean_kernel<<<x->nlist, 256, 0, st>>>(x->xpm, x->d_pad, x->list_off, mscale, d_s, lcent);
  ADN_LAUNCH("list_mean_kernel");
  return ADANNS_OK;
}

// rows[i] -= lcent[assign[ids[i]]] for n rows of ldr floats (first d_s)
__global__ void sub_list_centre_kernel(float *__restrict__ rows, int64_t n, int ldr, int d_s,
                                       const int64_t *__restrict__ ids64,
                                       const int32_t *__restrict__ ids32,
                                       const int32_t *__restrict__ assign,
                                       const float *__restrict__ lcent) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * d_s) return;
  const int64_t i = e / d_s;
  const int j = (int)(e % d_s);
  const int64_t id = ids64 ? ids64[i] : (int64_t)ids32[i];
  rows[i * ldr + j] -= lcent[(int64_t)assign[id] * d_s + j];
}

int launch_sub_list_centre(float *rows, int64_t n, int ldr, int d_s, const int64_t *ids64,
                           const int32_t *ids32, const int32_t *assign, const float *lcent,
                           cudaStream_t st) {
  if (n <= 0) return ADANNS_OK;
  sub_list_centre_kernel<<<(unsigned)((n * d_s + 255) / 256), 256, 0, st>>>(
      rows, n, ldr, d_s, ids64, ids32, assign, lcent);
  ADN_LAUNCH("sub_list_centre_kernel");
  return ADANNS_OK;
}

// S[l][m][c] = 2 <w_l,m, C_m[c]> and w2[l] = |w_l|^2; grid (nlist, M), c = thread
__global__ void residual_tables_kernel(const float *__restrict__ w, int d_s, int M, int dsub,
                                       const float *__restrict__ C, float *__restrict__ S,
                                       float *__restrict__ w2) {
  const int l = blockIdx.x, m = blockIdx.y, c = threadIdx.x;
  const float *wl = w + (int64_t)l * d_s + m * dsub;
  const float *cw = C + ((int64_t)m * 256 + c) * dsub;
  float acc = 0.f;
  for (int t = 0; t < dsub; ++t) acc = fmaf(wl[t], cw[t], acc);
  S[((int64_t)l * M + m) * 256 + c] = 2.f * acc;
  if (m == 0 && c == 0) {
    float s2 = 0.f;
    for (int t = 0; t < d_s; ++t) s2 = fmaf(w[(int64_t)l * d_s + t], w[(int64_t)l * d_s + t], s2);
    w2[l] = s2;
  }
}

int launch_residual_tables(const float *w, int nlist, int d_s, int M, const float *C, float *S,
                           float *w2, cudaStream_t st) {
  residual_tables_kernel<<<dim3(nlist, M), 256, 0, st>>>(w, d_s, M, d_s / M, C, S, w2);
  ADN_LAUNCH("residual_tables_kernel");
  return ADANNS_OK;
}

}  // namespace adn
