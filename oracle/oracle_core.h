/* FP64 CPU oracle (test infrastructure only; see oracle_core.c). */
#ifndef ORACLE_CORE_H
#define ORACLE_CORE_H
#include <stdint.h>

uint64_t orc_splitmix64_next(uint64_t *state);
int orc_sample(uint64_t seed, int64_t n, int64_t take, int64_t *out);
void orc_prefix_normalize(const float *x, int64_t n, int64_t ld, int m, int normalize,
                          double *out);
void orc_assign(const double *T, int64_t n, int dim, const double *C, int nc, int32_t *a,
                double *best, double *second, int nthreads);
int orc_ivf_search(const float *db, int64_t N, int d, const float *cent, int nlist, int ldc,
                   const int64_t *list_off, const int32_t *list_ids, const float *queries,
                   int64_t B, int d_c, int d_s, int nprobe, int k_out, int normalize,
                   int64_t *out_ids, double *out_dist, int32_t *out_probes, double *out_pdist,
                   int64_t *out_ncand, int nthreads);
int orc_pq_encode(const float *x, int64_t n, int64_t ld, int d_s, int M, int normalize,
                  const double *R, const double *C, const float *lcent, const int32_t *assign,
                  uint8_t *codes, int nthreads);
int orc_ivfopq_search(const float *db, int64_t N, int d, const float *cent, int nlist, int ldc,
                      const int64_t *list_off, const int32_t *list_ids, const float *R,
                      const float *codebooks, const uint8_t *codes, int M,
                      const float *queries, int64_t B, int d_c, int d_s, int nprobe, int k_out,
                      int rerank_k, int normalize, const float *lcent, int64_t *out_ids,
                      double *out_dist, int32_t *out_probes, double *out_pdist, int nthreads);
#endif
