// Index files: adanns_index_export / adanns_index_import.
//
// An AdANNS index is formed once and then serves many queries (Sec. 5
// "Search for AdANNS Hyperparameters"), so it is written to a file once and
// loaded by later processes instead of being rebuilt.  The file holds what
// defines the index -- the FP32 centroids, every row's list, the database rows
// in id order and the OPQ data -- and import re-creates the derived layouts
// (prefix-major lists, inverse prefix norms, low-precision tiers, centroid
// tables) with the same code adanns_index_create runs, so an imported index
// searches bit-identically to the exported one.
//
// Layout (little-endian): a 96-byte header (FileHeader), then
//   float   centroids[nlist][d_c]
//   int32   assign[N]               list of each database id
//   float   rows[N][d]              database rows, id order
//   if opq_M > 0:
//   float   R[opq_ds][opq_ds]       z = x R
//   float   codebooks[opq_M][256][opq_ds / opq_M]
//   uint8   codes[N][opq_M]         id order
//   if opq_flags & 1 (residual codes):
//   float   list_centres[nlist][opq_ds]
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace adn {
namespace {

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t N;
  int32_t d, d_c, nlist, metric, storage, opq_ds, opq_M, opq_flags;
  int32_t reserved[10];
};
static_assert(sizeof(FileHeader) == 96, "file header is 96 bytes");
constexpr char kMagic[8] = {'A', 'D', 'A', 'N', 'N', 'S', 'I', 'X'};
constexpr uint32_t kVersion = 1;
constexpr int64_t CHUNK_BYTES = 64ll << 20;  // rows moved per host <-> device copy

// rows [i0, i0 + n) of the database in id order, out of the prefix-major lists
// (one warp per row)
__global__ void rows_from_lists_kernel(const float *__restrict__ xpm, int d, int d_pad,
                                       const int64_t *__restrict__ list_off,
                                       const int32_t *__restrict__ assign,
                                       const int32_t *__restrict__ pos_of_id, int64_t i0,
                                       int64_t n, float *__restrict__ out) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int64_t id = i0 + w;
  const int l = assign[id];
  const int64_t off = list_off[l];
  const int64_t nl = list_off[l + 1] - off;
  const int64_t m = pos_of_id[id] - off;
  const float *src = xpm + off * d_pad;
  for (int j = lane; j < d; j += 32)
    out[w * d + j] = src[(int64_t)(j >> 4) * 16 * nl + m * 16 + (j & 15)];
}

// codes of ids [i0, i0 + n) out of the list-order code table
__global__ void codes_by_id_kernel(const uint8_t *__restrict__ codes, const int32_t *__restrict__ pos_of_id,
                                   int64_t i0, int64_t n, int M, uint8_t *__restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * M) return;
  const int64_t r = e / M;
  out[e] = codes[(int64_t)pos_of_id[i0 + r] * M + e % M];
}

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

int write_all(FILE *f, const void *p, size_t bytes, const char *what) {
  if (bytes && fwrite(p, 1, bytes, f) != bytes)
    return fail(ADANNS_ERR_ARG, std::string("index file: writing ") + what + " failed");
  return ADANNS_OK;
}

int read_all(FILE *f, void *p, size_t bytes, const char *what) {
  if (bytes && fread(p, 1, bytes, f) != bytes)
    return fail(ADANNS_ERR_STATE, std::string("index file: truncated in ") + what);
  return ADANNS_OK;
}

// device -> file through a host buffer
int dev_to_file(FILE *f, const void *dev, size_t bytes, cudaStream_t st, const char *what) {
  std::vector<unsigned char> h(bytes);
  ADN_CUDA(cudaMemcpyAsync(h.data(), dev, bytes, cudaMemcpyDeviceToHost, st));
  ADN_CUDA(cudaStreamSynchronize(st));
  return write_all(f, h.data(), bytes, what);
}

// file -> fresh device allocation (caller frees)
template <class T>
int file_to_dev(FILE *f, T **dev, size_t count, cudaStream_t st, const char *what) {
  *dev = nullptr;
  const size_t bytes = count * sizeof(T);
  if (cudaMalloc((void **)dev, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    *dev = nullptr;
    return fail(ADANNS_ERR_OOM, std::string("index import: device allocation for ") + what);
  }
  std::vector<unsigned char> h((size_t)std::min<int64_t>((int64_t)bytes, CHUNK_BYTES));
  for (size_t o = 0; o < bytes; o += h.size()) {
    const size_t b = std::min(h.size(), bytes - o);
    int rc;
    if ((rc = read_all(f, h.data(), b, what))) return rc;
    ADN_CUDA(cudaMemcpyAsync((unsigned char *)*dev + o, h.data(), b, cudaMemcpyHostToDevice, st));
    ADN_CUDA(cudaStreamSynchronize(st));  // the host buffer is reused
  }
  return ADANNS_OK;
}

struct DevBufs {
  void *p[8] = {nullptr};
  int n = 0;
  ~DevBufs() {
    for (int i = 0; i < n; ++i) cudaFree(p[i]);
  }
  template <class T>
  void keep(T *q) { p[n++] = (void *)q; }
};

}  // namespace
}  // namespace adn

using namespace adn;

extern "C" int adanns_index_export(const adanns_index *idx, const char *path, void *cuda_stream) {
  if (!idx || !path) return fail(ADANNS_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  File file;
  file.f = fopen(path, "wb");
  if (!file.f) return fail(ADANNS_ERR_ARG, std::string("cannot open ") + path + " for writing");
  FileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(FileHeader);
  h.N = idx->N;
  h.d = idx->d;
  h.d_c = idx->d_c;
  h.nlist = idx->nlist;
  h.metric = idx->metric;
  h.storage = idx->storage;
  h.opq_ds = idx->codes ? idx->opq_ds : 0;
  h.opq_M = idx->codes ? idx->opq_M : 0;
  h.opq_flags = idx->codes && idx->opq_lcent ? 1 : 0;
  int rc;
  if ((rc = write_all(file.f, &h, sizeof(h), "the header"))) return rc;
  if ((rc = dev_to_file(file.f, idx->centroids, sizeof(float) * idx->nlist * idx->d_c, st,
                        "the centroids")) ||
      (rc = dev_to_file(file.f, idx->assign, sizeof(int32_t) * idx->N, st, "the assignment")))
    return rc;
  // rows in id order, chunk by chunk
  const int64_t rows = std::max<int64_t>(1, CHUNK_BYTES / (4 * (int64_t)idx->d));
  Scratch s(st);
  float *buf;
  if ((rc = s.get(&buf, (size_t)std::min(rows, idx->N) * idx->d))) return rc;
  std::vector<float> hb((size_t)std::min(rows, idx->N) * idx->d);
  for (int64_t i0 = 0; i0 < idx->N; i0 += rows) {
    const int64_t n = std::min(rows, idx->N - i0);
    rows_from_lists_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(
        idx->xpm, idx->d, idx->d_pad, idx->list_off, idx->assign, idx->pos_of_id, i0, n, buf);
    ADN_LAUNCH("rows_from_lists_kernel");
    ADN_CUDA(cudaMemcpyAsync(hb.data(), buf, sizeof(float) * n * idx->d, cudaMemcpyDeviceToHost, st));
    ADN_CUDA(cudaStreamSynchronize(st));
    if ((rc = write_all(file.f, hb.data(), sizeof(float) * n * idx->d, "the rows"))) return rc;
  }
  if (h.opq_M > 0) {
    const int M = h.opq_M, ds = h.opq_ds;
    if ((rc = dev_to_file(file.f, idx->opq_R, sizeof(float) * ds * ds, st, "the rotation")) ||
        (rc = dev_to_file(file.f, idx->opq_C, sizeof(float) * M * 256 * (ds / M), st,
                          "the codebooks")))
      return rc;
    const int64_t crow = std::max<int64_t>(1, CHUNK_BYTES / M);
    uint8_t *cb;
    if ((rc = s.get(&cb, (size_t)std::min(crow, idx->N) * M))) return rc;
    std::vector<uint8_t> hc((size_t)std::min(crow, idx->N) * M);
    for (int64_t i0 = 0; i0 < idx->N; i0 += crow) {
      const int64_t n = std::min(crow, idx->N - i0);
      codes_by_id_kernel<<<(unsigned)((n * M + 255) / 256), 256, 0, st>>>(idx->codes, idx->pos_of_id,
                                                                         i0, n, M, cb);
      ADN_LAUNCH("codes_by_id_kernel");
      ADN_CUDA(cudaMemcpyAsync(hc.data(), cb, (size_t)n * M, cudaMemcpyDeviceToHost, st));
      ADN_CUDA(cudaStreamSynchronize(st));
      if ((rc = write_all(file.f, hc.data(), (size_t)n * M, "the codes"))) return rc;
    }
    if ((h.opq_flags & 1) &&
        (rc = dev_to_file(file.f, idx->opq_lcent, sizeof(float) * idx->nlist * ds, st,
                          "the list centres")))
      return rc;
  }
  if (fflush(file.f) != 0) return fail(ADANNS_ERR_ARG, "index file: flush failed");
  return ADANNS_OK;
}

extern "C" int adanns_index_import(const char *path, void *cuda_stream, adanns_index **out) {
  if (!path || !out) return fail(ADANNS_ERR_ARG, "NULL argument");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  File file;
  file.f = fopen(path, "rb");
  if (!file.f) return fail(ADANNS_ERR_ARG, std::string("cannot open ") + path);
  FileHeader h;
  int rc;
  if ((rc = read_all(file.f, &h, sizeof(h), "the header"))) return rc;
  if (memcmp(h.magic, kMagic, 8) != 0) return fail(ADANNS_ERR_STATE, "not an AdANNS index file");
  if (h.version != kVersion || h.header_bytes != sizeof(FileHeader))
    return fail(ADANNS_ERR_STATE, "unsupported index file version " + std::to_string(h.version));
  if (h.N < 1 || h.N > INT32_MAX || h.d < 1 || h.nlist < 1 || h.nlist > 32768 || h.d_c < 1 ||
      h.d_c > h.d || h.opq_M < 0 || (h.opq_M > 0 && (h.opq_ds < 1 || h.opq_ds % h.opq_M != 0)) ||
      (h.opq_flags & ~1) != 0 || (h.opq_flags && h.opq_M == 0))
    return fail(ADANNS_ERR_STATE, "index file header holds inconsistent sizes");
  DevBufs tmp;
  float *cent, *rows, *R = nullptr, *C = nullptr, *lc = nullptr;
  int32_t *assign;
  uint8_t *codes = nullptr;
  rc = file_to_dev(file.f, &cent, (size_t)h.nlist * h.d_c, st, "the centroids");
  tmp.keep(cent);
  if (rc) return rc;
  rc = file_to_dev(file.f, &assign, (size_t)h.N, st, "the assignment");
  tmp.keep(assign);
  if (rc) return rc;
  rc = file_to_dev(file.f, &rows, (size_t)h.N * h.d, st, "the rows");
  tmp.keep(rows);
  if (rc) return rc;
  if (h.opq_M > 0) {
    rc = file_to_dev(file.f, &R, (size_t)h.opq_ds * h.opq_ds, st, "the rotation");
    tmp.keep(R);
    if (rc) return rc;
    rc = file_to_dev(file.f, &C, (size_t)h.opq_M * 256 * (h.opq_ds / h.opq_M), st, "the codebooks");
    tmp.keep(C);
    if (rc) return rc;
    rc = file_to_dev(file.f, &codes, (size_t)h.N * h.opq_M, st, "the codes");
    tmp.keep(codes);
    if (rc) return rc;
    if (h.opq_flags & 1) {
      rc = file_to_dev(file.f, &lc, (size_t)h.nlist * h.opq_ds, st, "the list centres");
      tmp.keep(lc);
      if (rc) return rc;
    }
  }
  unsigned char extra;
  if (fread(&extra, 1, 1, file.f) != 0) return fail(ADANNS_ERR_STATE, "index file is longer than its header says");
  adanns_index *idx = nullptr;
  if ((rc = adanns_index_create(rows, h.N, h.d, cent, h.nlist, h.d_c, assign, h.metric, h.storage,
                                cuda_stream, &idx)))
    return rc;
  if (h.opq_M > 0 &&
      (rc = (h.opq_flags & 1)
                ? adanns_index_set_opq_residual(idx, h.opq_ds, h.opq_M, R, C, codes, lc, cuda_stream)
                : adanns_index_set_opq(idx, h.opq_ds, h.opq_M, R, C, codes, cuda_stream))) {
    adanns_index_free(idx);
    return rc;
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    adanns_index_free(idx);
    return cuda_fail(e, "index import");
  }
  *out = idx;
  return ADANNS_OK;
}
