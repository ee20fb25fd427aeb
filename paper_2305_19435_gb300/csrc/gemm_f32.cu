// FP32 GEMM for the OPQ rotation steps (Sec. 3 "OPQ": z = x R, the Procrustes
// product Y^T Zhat and the polar iteration).  C = alpha * op(A) * B + beta * C,
// op(A) = A or A^T, all row-major with explicit leading dimensions.  64 x 64
// output tiles, K in steps of 16, each of 256 threads accumulating 4 x 4 in
// FP32 FFMA.  Large K is split over CTAs (split-K) with FP32 atomics into C;
// the caller then owns a C that was pre-scaled by beta.
#include <algorithm>

#include "internal.cuh"

namespace adn {

namespace {
constexpr int TM = 64, TN = 64, TK = 16;

template <bool TA>
__global__ void __launch_bounds__(256) gemm_f32_kernel(int M, int N, int K, float alpha,
                                                        const float *__restrict__ A, int lda,
                                                        const float *__restrict__ B, int ldb,
                                                        float *__restrict__ C, int ldc, int kslice,
                                                        bool atomic_out) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int k_beg = blockIdx.z * kslice;
  const int k_end = min(K, k_beg + kslice);
  float acc[4][4] = {};
  for (int k0 = k_beg; k0 < k_end; k0 += TK) {
    // A tile: TM x TK elements of op(A)
    for (int e = tid; e < TM * TK; e += 256) {
      int mm, kk;
      if (TA) { kk = e / TM; mm = e % TM; } else { mm = e / TK; kk = e % TK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < k_end) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = tid; e < TK * TN; e += 256) {
      const int kk = e / TN, nn = e % TN;
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < k_end && gn < N) ? B[(int64_t)gk * ldb + gn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) {
        float *c = C + (int64_t)gm * ldc + gn;
        if (atomic_out) atomicAdd(c, alpha * acc[i][j]);
        else *c = alpha * acc[i][j] + *c;
      }
    }
}

__global__ void scale_kernel(float *C, int M, int N, int ldc, float beta) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  const int i = (int)(e / N), j = (int)(e % N);
  float *c = C + (int64_t)i * ldc + j;
  *c = beta == 0.f ? 0.f : beta * *c;
}
}  // namespace

int launch_gemm_f32(bool transA, int M, int N, int K, float alpha, const float *A, int lda,
                    const float *B, int ldb, float beta, float *C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return ADANNS_OK;
  const int64_t mn = (int64_t)M * N;
  scale_kernel<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(C, M, N, ldc, beta);
  ADN_LAUNCH("scale_kernel");
  if (K <= 0) return ADANNS_OK;
  const int gx = (N + TN - 1) / TN, gy = (M + TM - 1) / TM;
  // split K so that the grid covers the GPU when the output is small
  int splits = 1;
  const int tiles = gx * gy;
  const int target = 2 * num_sms();
  if (tiles < target) splits = std::max(1, std::min((K + 1023) / 1024, target / tiles));
  int kslice = (K + splits - 1) / splits;
  kslice = (kslice + TK - 1) / TK * TK;
  splits = (K + kslice - 1) / kslice;
  dim3 grid(gx, gy, splits);
  const bool atomic_out = true;  // C was pre-scaled by beta above
  if (transA)
    gemm_f32_kernel<true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, C, ldc, kslice,
                                                atomic_out);
  else
    gemm_f32_kernel<false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, C, ldc, kslice,
                                                 atomic_out);
  ADN_LAUNCH("gemm_f32_kernel");
  return ADANNS_OK;
}

}  // namespace adn
