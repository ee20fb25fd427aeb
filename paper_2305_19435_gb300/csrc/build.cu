// Index construction kernels (Algorithm 1 adannsConstruction; Sec. 3 "IVF"):
// prefix normalisation of the training sample, the Lloyd update with FP64
// centroid sums, the stable CSR inverted-list build (counting sort that keeps
// ids ascending inside each list), the prefix-major re-layout of the vectors
// and the per-granularity inverse prefix norms.
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"

namespace adn {


// rows[r] (or r) of x, first `dim` coordinates, times 1/||x[0:dim]|| (metric
// L2_PREFIXNORM) into out (rows of ldo, zero padded).  One warp per row.
__global__ void gather_normalize_kernel(const float *__restrict__ x, int64_t n, int ld,
                                        const int64_t *__restrict__ rows, int dim, int metric,
                                        float *__restrict__ out, int ldo) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const float *src = x + (rows ? rows[r] : r) * (int64_t)ld;
  float s = 0.f;
  for (int j = lane; j < dim; j += 32) s = fmaf(src[j], src[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  float nu = 1.f;
  if (metric == ADANNS_METRIC_L2_PREFIXNORM) nu = s > 0.f ? 1.f / sqrtf(s) : 0.f;
  for (int j = lane; j < ldo; j += 32) out[r * ldo + j] = j < dim ? src[j] * nu : 0.f;
}

int launch_gather_normalize(const float *x, int64_t n, int ld, const int64_t *rows, int dim,
                            int metric, float *out, int ldo, cudaStream_t st) {
  if (n <= 0) return ADANNS_OK;
  gather_normalize_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(x, n, ld, rows, dim, metric,
                                                                  out, ldo);
  ADN_LAUNCH("gather_normalize_kernel");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- Lloyd update
__global__ void km_accum_kernel(const float *__restrict__ t, int64_t n, int ld, int dim,
                                const int32_t *__restrict__ assign, int nc,
                                double *__restrict__ sums, int32_t *__restrict__ counts) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * dim) return;
  const int64_t i = e / dim;
  const int j = (int)(e - i * dim);
  const int h = assign[i];
  if (h < 0 || h >= nc) return;  // out-of-range assignments are ignored
  atomicAdd(&sums[(int64_t)h * dim + j], (double)t[i * ld + j]);
  if (j == 0) atomicAdd(&counts[h], 1);
}

__global__ void km_finish_kernel(const double *__restrict__ sums, const int32_t *__restrict__ counts,
                                 int nc, int dim, float *__restrict__ cent) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nc * dim) return;
  const int h = (int)(e / dim);
  const int c = counts[h];
  if (c > 0) cent[e] = (float)(sums[e] / (double)c);
}

int launch_kmeans_update(const float *t, int64_t n, int ld, int dim, const int32_t *assign,
                         int nc, double *sums, int32_t *counts, float *cent, cudaStream_t st) {
  ADN_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)nc * dim, st));
  ADN_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)nc, st));
  const int64_t ne = n * dim;
  if (ne > 0) {
    km_accum_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(t, n, ld, dim, assign, nc,
                                                                  sums, counts);
    ADN_LAUNCH("km_accum_kernel");
  }
  const int64_t nce = (int64_t)nc * dim;
  km_finish_kernel<<<(unsigned)((nce + 255) / 256), 256, 0, st>>>(sums, counts, nc, dim, cent);
  ADN_LAUNCH("km_finish_kernel");
  return ADANNS_OK;
}

// objective: sum of the distances held in the keys' high words (FP64)
__global__ void sum_keys_kernel(const uint64_t *__restrict__ keys, int64_t n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    if (k != KEY_MAX) s += (double)__uint_as_float((uint32_t)(k >> 32));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

int launch_sum_keys(const uint64_t *keys, int64_t n, double *out, cudaStream_t st) {
  ADN_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  if (n <= 0) return ADANNS_OK;
  int g = (int)std::min<int64_t>((n + 255) / 256, 4 * num_sms());
  sum_keys_kernel<<<g, 256, 0, st>>>(keys, n, out);
  ADN_LAUNCH("sum_keys_kernel");
  return ADANNS_OK;
}

// number of assignments outside [0, nlist)
__global__ void count_bad_assign_kernel(const int32_t *__restrict__ a, int64_t n, int nlist,
                                        int *__restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (a[i] < 0 || a[i] >= nlist)) atomicAdd(bad, 1);
}

int check_assignment(const int32_t *a, int64_t n, int nlist, cudaStream_t st) {
  Scratch s(st);
  int *bad;
  int rc;
  if ((rc = s.get(&bad, 1))) return rc;
  ADN_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  if (n > 0) {
    count_bad_assign_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, nlist, bad);
    ADN_LAUNCH("count_bad_assign_kernel");
  }
  int h = 0;
  ADN_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  ADN_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(ADANNS_ERR_ARG, std::to_string(h) + " list assignments outside [0, nlist)");
  return ADANNS_OK;
}

// ---------------------------------------------------------------- CSR build
// Stable counting sort of ids by list: per-tile histograms (list-major), one
// exclusive scan over the flattened [list][tile] counts, then an in-order
// scatter inside each tile (warp match groups preserve id order).
constexpr int CSR_TILE = 4096;
constexpr int SCAN_BLOCK = 4096;

__global__ void csr_hist_kernel(const int32_t *__restrict__ a, int64_t N, int nlist, int ntile,
                                int32_t *__restrict__ counts) {
  extern __shared__ int32_t h[];
  for (int l = threadIdx.x; l < nlist; l += blockDim.x) h[l] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * CSR_TILE;
  // one atomic per distinct bucket in a warp (a heavily repeated bucket, e.g.
  // a padding bucket, would otherwise serialise on one shared address)
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < CSR_TILE; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const bool valid = base + i < N;
    const int l = valid ? a[base + i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[l], __popc(peers));
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nlist; l += blockDim.x)
    counts[(int64_t)l * ntile + blockIdx.x] = h[l];
}

// block-wise sums of v (SCAN_BLOCK elements per block)
__global__ void scan_reduce_kernel(const int32_t *__restrict__ v, int64_t n,
                                   int64_t *__restrict__ bsum) {
  __shared__ int64_t red[1024];
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  int64_t s = 0;
  for (int i = threadIdx.x; i < SCAN_BLOCK && base + i < n; i += blockDim.x) s += v[base + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = red[0];
}

// single CTA: exclusive scan of bsum in place
__global__ void scan_bsum_kernel(int64_t *__restrict__ bsum, int nb) {
  __shared__ int64_t s[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int64_t x = i < nb ? bsum[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int64_t y = (int)threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < nb) bsum[i] = carry + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
}

// exclusive scan inside each block, plus the block's offset; writes out[] as int32
__global__ void scan_apply_kernel(const int32_t *__restrict__ v, int64_t n,
                                  const int64_t *__restrict__ bsum, int32_t *__restrict__ out) {
  __shared__ int64_t s[1024];
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  // each thread owns 4 consecutive elements
  int64_t loc[4];
  int64_t tsum = 0;
  for (int u = 0; u < 4; ++u) {
    const int64_t i = base + threadIdx.x * 4 + u;
    loc[u] = i < n ? v[i] : 0;
    tsum += loc[u];
  }
  s[threadIdx.x] = tsum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t y = (int)threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += y;
    __syncthreads();
  }
  int64_t run = bsum[blockIdx.x] + s[threadIdx.x] - tsum;
  for (int u = 0; u < 4; ++u) {
    const int64_t i = base + threadIdx.x * 4 + u;
    if (i < n) out[i] = (int32_t)run;
    run += loc[u];
  }
}

__global__ void csr_offsets_kernel(const int32_t *__restrict__ scanned, int nlist, int ntile,
                                   int64_t N, int64_t *__restrict__ list_off) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < nlist) list_off[l] = scanned[(int64_t)l * ntile];
  if (l == nlist) list_off[nlist] = N;
}

// one warp per tile, elements in id order
__global__ void csr_scatter_kernel(const int32_t *__restrict__ a, int64_t N, int nlist, int ntile,
                                   const int32_t *__restrict__ scanned,
                                   int32_t *__restrict__ list_ids) {
  extern __shared__ int32_t run[];
  const int t = blockIdx.x, lane = threadIdx.x;
  for (int l = lane; l < nlist; l += 32) run[l] = scanned[(int64_t)l * ntile + t];
  __syncwarp();
  const int64_t base = (int64_t)t * CSR_TILE;
  const int64_t end = min(N, base + CSR_TILE);
  for (int64_t c = base; c < end; c += 32) {
    const int64_t i = c + lane;
    const bool valid = i < end;
    const int l = valid ? a[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & lanemask_lt());
    const int start = valid ? run[l] : 0;
    __syncwarp();
    if (valid) list_ids[start + rank] = (int32_t)i;
    if (valid && lane == leader) run[l] = start + __popc(peers);
    __syncwarp();
  }
}

// exclusive scan of n int32 counts (block sums, their scan, the per-block scan)
int launch_scan_i32(const int32_t *v, int64_t n, int32_t *out, cudaStream_t st) {
  if (n <= 0) return ADANNS_OK;
  const int nb = (int)((n + SCAN_BLOCK - 1) / SCAN_BLOCK);
  Scratch s(st);
  int64_t *bsum;
  int rc;
  if ((rc = s.get(&bsum, nb))) return rc;
  scan_reduce_kernel<<<nb, 1024, 0, st>>>(v, n, bsum);
  ADN_LAUNCH("scan_reduce_kernel");
  scan_bsum_kernel<<<1, 1024, 0, st>>>(bsum, nb);
  ADN_LAUNCH("scan_bsum_kernel");
  scan_apply_kernel<<<nb, 1024, 0, st>>>(v, n, bsum, out);
  ADN_LAUNCH("scan_apply_kernel");
  return ADANNS_OK;
}

int build_csr(const int32_t *assign, int64_t N, int nlist, int64_t *list_off, int32_t *list_ids,
              cudaStream_t st) {
  if (nlist > 32768) return fail(ADANNS_ERR_ARG, "nlist above 32768");
  const int ntile = (int)((N + CSR_TILE - 1) / CSR_TILE);
  const int64_t nc = (int64_t)nlist * ntile;
  const int nb = (int)((nc + SCAN_BLOCK - 1) / SCAN_BLOCK);
  Scratch s(st);
  int32_t *counts, *scanned;
  int64_t *bsum;
  int rc;
  if ((rc = s.get(&counts, nc)) || (rc = s.get(&scanned, nc)) || (rc = s.get(&bsum, nb))) return rc;
  const size_t hs = (size_t)nlist * 4;
  ADN_CUDA(ensure_smem((const void *)csr_hist_kernel, (size_t)(hs)));
  ADN_CUDA(ensure_smem((const void *)csr_scatter_kernel, (size_t)(hs)));
  if (ntile > 0) {
    csr_hist_kernel<<<ntile, 256, hs, st>>>(assign, N, nlist, ntile, counts);
    ADN_LAUNCH("csr_hist_kernel");
  }
  if (nc > 0) {
    scan_reduce_kernel<<<nb, 1024, 0, st>>>(counts, nc, bsum);
    ADN_LAUNCH("scan_reduce_kernel");
    scan_bsum_kernel<<<1, 1024, 0, st>>>(bsum, nb);
    ADN_LAUNCH("scan_bsum_kernel");
    scan_apply_kernel<<<nb, 1024, 0, st>>>(counts, nc, bsum, scanned);
    ADN_LAUNCH("scan_apply_kernel");
  }
  if (ntile > 0) {
    csr_offsets_kernel<<<(nlist + 1 + 255) / 256, 256, 0, st>>>(scanned, nlist, ntile, N, list_off);
    ADN_LAUNCH("csr_offsets_kernel");
    csr_scatter_kernel<<<ntile, 32, hs, st>>>(assign, N, nlist, ntile, scanned, list_ids);
    ADN_LAUNCH("csr_scatter_kernel");
  } else {
    ADN_CUDA(cudaMemsetAsync(list_off, 0, sizeof(int64_t) * (nlist + 1), st));
  }
  return ADANNS_OK;
}

// ---------------------------------------------------------------- prefix-major layout
// For member position p (list order) with id = list_ids[p] in list l:
//   xpm[off_l*d_pad + b*16*n_l + (p - off_l)*16 + j] = x[id][16b + j]  (0 beyond d).
// One warp per member; each lane moves 16-byte pieces.
__global__ void prefix_major_kernel(const float *__restrict__ x, int ld, int d, int d_pad,
                                    const int64_t *__restrict__ list_off,
                                    const int32_t *__restrict__ list_ids,
                                    const int32_t *__restrict__ assign, int64_t N,
                                    float *__restrict__ xpm) {
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= N) return;
  // NULL list_ids / assign / list_off: identity order, one list holding all N
  const int id = list_ids ? list_ids[p] : (int)p;
  const int l = assign ? assign[id] : 0;
  const int64_t off = list_off ? list_off[l] : 0;
  const int64_t nl = list_off ? list_off[l + 1] - off : N;
  const int64_t m = p - off;
  const float *src = x + (int64_t)id * ld;
  float *dst = xpm + off * d_pad + m * 16;
  const bool vec = (d % 4 == 0) && (ld % 4 == 0) && (((uintptr_t)x & 15) == 0);
  for (int c = lane; c < d_pad / 4; c += 32) {
    const int b = c >> 2, part = c & 3;
    const int j = c * 4;
    float4 v;
    if (vec && j + 3 < d) {
      v = *(const float4 *)(src + j);
    } else {
      v.x = j < d ? src[j] : 0.f;
      v.y = j + 1 < d ? src[j + 1] : 0.f;
      v.z = j + 2 < d ? src[j + 2] : 0.f;
      v.w = j + 3 < d ? src[j + 3] : 0.f;
    }
    *(float4 *)(dst + (int64_t)b * 16 * nl + part * 4) = v;
  }
}

int launch_prefix_major(const float *x, int ld, int d, int d_pad, const int64_t *list_off,
                        const int32_t *list_ids, const int32_t *assign, int64_t N, float *xpm,
                        cudaStream_t st) {
  if (N <= 0) return ADANNS_OK;
  prefix_major_kernel<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(x, ld, d, d_pad, list_off,
                                                              list_ids, assign, N, xpm);
  ADN_LAUNCH("prefix_major_kernel");
  return ADANNS_OK;
}

// pos[list_ids[p]] = p
__global__ void positions_kernel(const int32_t *__restrict__ list_ids, int64_t N,
                                 int32_t *__restrict__ pos) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) pos[list_ids[p]] = (int32_t)p;
}

int launch_positions(const int32_t *list_ids, int64_t N, int32_t *pos, cudaStream_t st) {
  if (N <= 0) return ADANNS_OK;
  positions_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(list_ids, N, pos);
  ADN_LAUNCH("positions_kernel");
  return ADANNS_OK;
}

// invn[g][p] = 1 / ||x[list_ids[p]][0:G[g]]|| (0 for a zero prefix; 1 for raw L2)
__global__ void inv_norms_kernel(const float *__restrict__ x, int ld, int d,
                                 const int32_t *__restrict__ list_ids, int64_t N, int metric,
                                 float *__restrict__ invn, int ng) {
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= N) return;
  const float *src = x + (int64_t)(list_ids ? list_ids[p] : p) * ld;
  for (int g = 0; g < ng; ++g) {
    const int m = kGranDev(g);
    float s = 0.f;
    for (int j = lane; j < m && j < d; j += 32) s = fmaf(src[j], src[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      float v = 1.f;
      if (metric == ADANNS_METRIC_L2_PREFIXNORM) v = s > 0.f ? 1.f / sqrtf(s) : 0.f;
      invn[(int64_t)g * N + p] = v;
    }
  }
}

int launch_inv_norms(const float *x, int ld, int d, const int32_t *list_ids, int64_t N, int metric,
                     float *invn, int ng, cudaStream_t st) {
  if (N <= 0) return ADANNS_OK;
  inv_norms_kernel<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(x, ld, d, list_ids, N, metric, invn,
                                                           ng);
  ADN_LAUNCH("inv_norms_kernel");
  return ADANNS_OK;
}

}  // namespace adn
