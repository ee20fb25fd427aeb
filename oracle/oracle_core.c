/*
 * FP64 CPU oracle for AdANNS-IVF and AdANNS-IVF-OPQ search (test infrastructure).
 *
 * This file is test infrastructure only.  It is called by the tests, by the
 * package smoke check and by the benchmark's CPU-baseline leg, never by the
 * GPU library, and it shares no code, header or table with it.  Everything is
 * written as the plain definition: no blocking, no fusion, no reordering.
 *
 * Arithmetic: inputs arrive as FP32 (the stored embeddings, the FP32 index
 * centroids / rotation / codebooks) and every computation runs in FP64.
 *
 * Sections followed:
 *  - Matryoshka prefixes: the first m coordinates of an MR form an m-dim
 *    representation (Sec. 3 "Matryoshka Representations").  A prefix used as a
 *    representation is L2-normalised at its own length:
 *    P_m(v) = v[0:m] / ||v[0:m]||, P_m(0) = 0.
 *  - IVF: Lloyd k-means coarse quantiser, inverted lists, nearest-centroid
 *    probing then an exhaustive scan of the probed lists (Sec. 3 "IVF").
 *  - AdANNS-IVF: cluster mapping with the d_c prefix, linear scan with the
 *    d_s prefix (Sec. 4.1, Algorithm 1, Table "formula" AdANNS-IVF row).
 *  - PQ / OPQ: m sub-vectors, 2^8 codewords each, search by m codebook
 *    lookups; OPQ learns an orthonormal rotation R first (Sec. 3 "OPQ").
 *  - AdANNS-IVFOPQ: IVF at d_c with OPQ distances on the d_s prefix inside the
 *    lists (Sec. 4.3, Table "formula" IVFOPQ row, read as asymmetric lookup).
 *  - Shortlist rerank with a higher-precision representation (Sec. 4.3).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle_core.h"

/* ------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea & Flood 2014; public-domain definition by   */
/* S. Vigna): state += golden gamma, then two xor-shift-multiply mixes. */
/* ------------------------------------------------------------------ */
uint64_t orc_splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* First `take` entries of a Fisher-Yates shuffle of [0, n): for i < take,
 * j = i + (next() mod (n - i)), swap(a[i], a[j]).  Returns 0, or -1 on bad
 * arguments / allocation failure. */
int orc_sample(uint64_t seed, int64_t n, int64_t take, int64_t *out) {
    if (n <= 0 || take < 0 || take > n) return -1;
    int64_t *a = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!a) return -1;
    for (int64_t i = 0; i < n; ++i) a[i] = i;
    uint64_t st = seed;
    for (int64_t i = 0; i < take; ++i) {
        uint64_t r = orc_splitmix64_next(&st);
        int64_t j = i + (int64_t)(r % (uint64_t)(n - i));
        int64_t t = a[i]; a[i] = a[j]; a[j] = t;
    }
    memcpy(out, a, sizeof(int64_t) * (size_t)take);
    free(a);
    return 0;
}

/* P_m of one FP32 row into FP64 (normalize != 0), or the raw prefix. */
static void prefix_of(const float *x, int m, int normalize, double *out) {
    for (int j = 0; j < m; ++j) out[j] = (double)x[j];
    if (!normalize) return;
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += out[j] * out[j];
    double nrm = sqrt(s);
    if (nrm == 0.0) {
        for (int j = 0; j < m; ++j) out[j] = 0.0;
    } else {
        for (int j = 0; j < m; ++j) out[j] = out[j] / nrm;
    }
}

void orc_prefix_normalize(const float *x, int64_t n, int64_t ld, int m, int normalize,
                          double *out) {
    for (int64_t i = 0; i < n; ++i) prefix_of(x + i * ld, m, normalize, out + i * (int64_t)m);
}

/* ---------------------------- threading ---------------------------- */
typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void *ctx; int64_t lo, hi; } range_job;

static void *range_thread(void *p) {
    range_job *j = (range_job *)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > n) nthreads = (int)(n > 0 ? n : 1);
    if (nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    range_job jobs[256];
    int started[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
        started[t] = pthread_create(&th[t], NULL, range_thread, &jobs[t]) == 0;
        if (!started[t]) fn(ctx, jobs[t].lo, jobs[t].hi);
    }
    for (int t = 0; t < nthreads; ++t)
        if (started[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ */
/* Lloyd assignment step (Sec. 3 "IVF"; Algorithm 1 constructClusters). */
/* a_t = argmin_h sum_j (T[t][j] - C[h][j])^2, ties -> smallest h.      */
/* best[t] = that minimum, second[t] = the runner-up distance.          */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *T; int dim; const double *C; int nc;
    int32_t *a; double *best; double *second;
} assign_ctx;

static void assign_range(void *p, int64_t lo, int64_t hi) {
    assign_ctx *c = (assign_ctx *)p;
    for (int64_t t = lo; t < hi; ++t) {
        const double *x = c->T + t * c->dim;
        double b = INFINITY, s = INFINITY;
        int32_t bi = -1;
        for (int h = 0; h < c->nc; ++h) {
            const double *mu = c->C + (int64_t)h * c->dim;
            double acc = 0.0;
            for (int j = 0; j < c->dim; ++j) {
                double diff = x[j] - mu[j];
                acc += diff * diff;
            }
            if (acc < b) { s = b; b = acc; bi = h; }
            else if (acc < s) { s = acc; }
        }
        c->a[t] = bi;
        if (c->best) c->best[t] = b;
        if (c->second) c->second[t] = s;
    }
}

void orc_assign(const double *T, int64_t n, int dim, const double *C, int nc, int32_t *a,
                double *best, double *second, int nthreads) {
    assign_ctx c = {T, dim, C, nc, a, best, second};
    parallel_for(n, nthreads, assign_range, &c);
}

/* ------------------------------------------------------------------ */
/* candidate ordering: by (distance, id) ascending                      */
/* ------------------------------------------------------------------ */
typedef struct { double dist; int64_t id; } cand;

static int cand_cmp(const void *pa, const void *pb) {
    const cand *a = (const cand *)pa, *b = (const cand *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* Cluster mapping (Algorithm 1 computeDistances + sortAscending[:n_p]):
 * D_h = sum_{j<d_c} (P_dc(q)_j - mu_h[j])^2, probes = the n_p smallest by
 * (D_h, h).  `cent` holds nlist rows of `ldc` FP32 values, of which the first
 * d_c are used.  Fills probes[0:nprobe] and pdist[0:min(nprobe+1,nlist)]. */
static void cluster_map(const float *q, int d_c, int normalize, const float *cent, int nlist,
                        int ldc, int nprobe, int32_t *probes, double *pdist, double *qbuf,
                        cand *cbuf) {
    prefix_of(q, d_c, normalize, qbuf);
    for (int h = 0; h < nlist; ++h) {
        double acc = 0.0;
        for (int j = 0; j < d_c; ++j) {
            double diff = qbuf[j] - (double)cent[(int64_t)h * ldc + j];
            acc += diff * diff;
        }
        cbuf[h].dist = acc;
        cbuf[h].id = h;
    }
    qsort(cbuf, (size_t)nlist, sizeof(cand), cand_cmp);
    for (int i = 0; i < nprobe; ++i) probes[i] = (int32_t)cbuf[i].id;
    int np1 = nprobe + 1 < nlist ? nprobe + 1 : nlist;
    if (pdist)
        for (int i = 0; i < np1; ++i) pdist[i] = cbuf[i].dist;
}

/* dist_m(q, x) = sum_{j<m} (P_m(q)_j - P_m(x)_j)^2, with P_m(q) given. */
static double scan_dist(const double *qs, const float *x, int m, int normalize, double *xbuf) {
    prefix_of(x, m, normalize, xbuf);
    double acc = 0.0;
    for (int j = 0; j < m; ++j) {
        double diff = qs[j] - xbuf[j];
        acc += diff * diff;
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* AdANNS-IVF search (Algorithm 1 adannsInference; Table "formula").     */
/* ------------------------------------------------------------------ */
typedef struct {
    const float *db; int64_t N; int d;
    const float *cent; int nlist; int ldc;
    const int64_t *off; const int32_t *ids;
    const float *queries; int d_c, d_s, nprobe, k_out, normalize;
    int64_t *out_ids; double *out_dist; int32_t *out_probes; double *out_pdist;
    int64_t *out_ncand; int pstride;
} ivf_ctx;

static void ivf_range(void *p, int64_t lo, int64_t hi) {
    ivf_ctx *c = (ivf_ctx *)p;
    int dmax = c->d;
    double *qbuf = (double *)malloc(sizeof(double) * (size_t)dmax);
    double *qs = (double *)malloc(sizeof(double) * (size_t)dmax);
    double *xbuf = (double *)malloc(sizeof(double) * (size_t)dmax);
    cand *cbuf = (cand *)malloc(sizeof(cand) * (size_t)c->nlist);
    int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->nprobe);
    for (int64_t qi = lo; qi < hi; ++qi) {
        const float *q = c->queries + qi * c->d;
        double *pd = c->out_pdist ? c->out_pdist + qi * c->pstride : NULL;
        cluster_map(q, c->d_c, c->normalize, c->cent, c->nlist, c->ldc, c->nprobe, probes, pd,
                    qbuf, cbuf);
        if (c->out_probes)
            for (int i = 0; i < c->nprobe; ++i) c->out_probes[qi * c->nprobe + i] = probes[i];
        int64_t ncand = 0;
        for (int i = 0; i < c->nprobe; ++i) ncand += c->off[probes[i] + 1] - c->off[probes[i]];
        cand *cs = (cand *)malloc(sizeof(cand) * (size_t)(ncand > 0 ? ncand : 1));
        prefix_of(q, c->d_s, c->normalize, qs);
        int64_t w = 0;
        for (int i = 0; i < c->nprobe; ++i) {
            int l = probes[i];
            for (int64_t p2 = c->off[l]; p2 < c->off[l + 1]; ++p2) {
                int64_t id = c->ids[p2];
                cs[w].dist = scan_dist(qs, c->db + id * c->d, c->d_s, c->normalize, xbuf);
                cs[w].id = id;
                ++w;
            }
        }
        qsort(cs, (size_t)w, sizeof(cand), cand_cmp);
        for (int r = 0; r < c->k_out; ++r) {
            if (r < w) {
                c->out_ids[qi * c->k_out + r] = cs[r].id;
                c->out_dist[qi * c->k_out + r] = cs[r].dist;
            } else {
                c->out_ids[qi * c->k_out + r] = -1;
                c->out_dist[qi * c->k_out + r] = INFINITY;
            }
        }
        if (c->out_ncand) c->out_ncand[qi] = w;
        free(cs);
    }
    free(qbuf); free(qs); free(xbuf); free(cbuf); free(probes);
}

int orc_ivf_search(const float *db, int64_t N, int d, const float *cent, int nlist, int ldc,
                   const int64_t *list_off, const int32_t *list_ids, const float *queries,
                   int64_t B, int d_c, int d_s, int nprobe, int k_out, int normalize,
                   int64_t *out_ids, double *out_dist, int32_t *out_probes, double *out_pdist,
                   int64_t *out_ncand, int nthreads) {
    if (d_c < 1 || d_c > ldc || d_s < 1 || d_s > d || nprobe < 1 || nprobe > nlist || k_out < 1)
        return -1;
    ivf_ctx c = {db, N, d, cent, nlist, ldc, list_off, list_ids, queries, d_c, d_s, nprobe,
                 k_out, normalize, out_ids, out_dist, out_probes, out_pdist, out_ncand,
                 nprobe + 1};
    parallel_for(B, nthreads, ivf_range, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* PQ encoding of the rotated, normalised d_s prefix (Sec. 3 "OPQ"):    */
/* z = P_ds(x) R, code[m] = argmin_c ||z_m - C_m[c]||^2, ties -> min c.  */
/* R is d_s x d_s row-major (z_j = sum_i x_i R[i][j]); C is M x 256 x   */
/* dsub.  Both are passed as FP64 arrays.                                */
/* ------------------------------------------------------------------ */
static void rotate(const double *xs, int d_s, const double *R, double *z) {
    for (int j = 0; j < d_s; ++j) z[j] = 0.0;
    for (int i = 0; i < d_s; ++i) {
        double xi = xs[i];
        const double *Ri = R + (int64_t)i * d_s;
        for (int j = 0; j < d_s; ++j) z[j] += xi * Ri[j];
    }
}

typedef struct {
    const float *x; int64_t ld; int d_s, M, normalize;
    const double *R, *C; uint8_t *codes;
    const float *lcent; const int32_t *assign;
} enc_ctx;

static void enc_range(void *p, int64_t lo, int64_t hi) {
    enc_ctx *c = (enc_ctx *)p;
    int dsub = c->d_s / c->M;
    double *xs = (double *)malloc(sizeof(double) * (size_t)c->d_s);
    double *z = (double *)malloc(sizeof(double) * (size_t)c->d_s);
    for (int64_t i = lo; i < hi; ++i) {
        prefix_of(c->x + i * c->ld, c->d_s, c->normalize, xs);
        if (c->lcent) {   /* residual: subtract the row's list centroid */
            const float *cl = c->lcent + (int64_t)c->assign[i] * c->d_s;
            for (int j = 0; j < c->d_s; ++j) xs[j] -= (double)cl[j];
        }
        rotate(xs, c->d_s, c->R, z);
        for (int m = 0; m < c->M; ++m) {
            double best = INFINITY;
            int bc = 0;
            for (int cc = 0; cc < 256; ++cc) {
                const double *cw = c->C + ((int64_t)m * 256 + cc) * dsub;
                double acc = 0.0;
                for (int t = 0; t < dsub; ++t) {
                    double diff = z[m * dsub + t] - cw[t];
                    acc += diff * diff;
                }
                if (acc < best) { best = acc; bc = cc; }
            }
            c->codes[i * c->M + m] = (uint8_t)bc;
        }
    }
    free(xs); free(z);
}

int orc_pq_encode(const float *x, int64_t n, int64_t ld, int d_s, int M, int normalize,
                  const double *R, const double *C, const float *lcent, const int32_t *assign,
                  uint8_t *codes, int nthreads) {
    if (M < 1 || d_s % M != 0 || (lcent && !assign)) return -1;
    enc_ctx c = {x, ld, d_s, M, normalize, R, C, codes, lcent, assign};
    parallel_for(n, nthreads, enc_range, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* AdANNS-IVFOPQ search with optional exact rerank of the ADC shortlist. */
/* ADC: LUT[m][c] = ||z_m - C_m[c]||^2 with z = P_ds(q) R; a member's    */
/* distance is sum_m LUT[m][code[m]] (m codebook lookups, Sec. 3).       */
/* Rerank: the rerank_k best by ADC are re-scored with dist_ds (FP64)    */
/* and the k_out best of those are returned (Sec. 4.3 shortlist-rerank). */
/* R, codebooks are the FP32 index values; codes are indexed by db id.   */
/* ------------------------------------------------------------------ */
typedef struct {
    const float *db; int d;
    const float *cent; int nlist; int ldc;
    const int64_t *off; const int32_t *ids;
    const float *R; const float *C; const uint8_t *codes; int M;
    const float *queries; int d_c, d_s, nprobe, k_out, rerank_k, normalize;
    int64_t *out_ids; double *out_dist; int32_t *out_probes; double *out_pdist; int pstride;
    const float *lcent;   /* residual codes: list centroids [nlist][d_s], else NULL */
} opq_ctx;

/* lut[m][c] = ||v_m - C_m[c]||^2 for the rotated vector v */
static void build_lut(const double *v, const float *C, int M, int dsub, double *lut) {
    for (int m = 0; m < M; ++m)
        for (int cc = 0; cc < 256; ++cc) {
            const float *cw = C + ((int64_t)m * 256 + cc) * dsub;
            double acc = 0.0;
            for (int t = 0; t < dsub; ++t) {
                double diff = v[m * dsub + t] - (double)cw[t];
                acc += diff * diff;
            }
            lut[m * 256 + cc] = acc;
        }
}

static void opq_range(void *p, int64_t lo, int64_t hi) {
    opq_ctx *c = (opq_ctx *)p;
    int dsub = c->d_s / c->M;
    double *qbuf = (double *)malloc(sizeof(double) * (size_t)c->d);
    double *qs = (double *)malloc(sizeof(double) * (size_t)c->d);
    double *z = (double *)malloc(sizeof(double) * (size_t)c->d);
    double *xbuf = (double *)malloc(sizeof(double) * (size_t)c->d);
    double *lut = (double *)malloc(sizeof(double) * (size_t)c->M * 256);
    cand *cbuf = (cand *)malloc(sizeof(cand) * (size_t)c->nlist);
    int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->nprobe);
    for (int64_t qi = lo; qi < hi; ++qi) {
        const float *q = c->queries + qi * c->d;
        double *pd = c->out_pdist ? c->out_pdist + qi * c->pstride : NULL;
        cluster_map(q, c->d_c, c->normalize, c->cent, c->nlist, c->ldc, c->nprobe, probes, pd,
                    qbuf, cbuf);
        if (c->out_probes)
            for (int i = 0; i < c->nprobe; ++i) c->out_probes[qi * c->nprobe + i] = probes[i];
        prefix_of(q, c->d_s, c->normalize, qs);
        for (int j = 0; j < c->d_s; ++j) {
            double acc = 0.0;
            for (int i = 0; i < c->d_s; ++i) acc += qs[i] * (double)c->R[(int64_t)i * c->d_s + j];
            z[j] = acc;
        }
        if (!c->lcent) build_lut(z, c->C, c->M, dsub, lut);
        int64_t ncand = 0;
        for (int i = 0; i < c->nprobe; ++i) ncand += c->off[probes[i] + 1] - c->off[probes[i]];
        cand *cs = (cand *)malloc(sizeof(cand) * (size_t)(ncand > 0 ? ncand : 1));
        int64_t w = 0;
        for (int i = 0; i < c->nprobe; ++i) {
            int l = probes[i];
            if (c->lcent) {
                /* residual codes: the query's rotated residual to list l,
                   (P_ds(q) - c_l) R, gives this list's lookup table */
                const float *cl = c->lcent + (int64_t)l * c->d_s;
                for (int j = 0; j < c->d_s; ++j) xbuf[j] = qs[j] - (double)cl[j];
                for (int j = 0; j < c->d_s; ++j) {
                    double acc = 0.0;
                    for (int t = 0; t < c->d_s; ++t)
                        acc += xbuf[t] * (double)c->R[(int64_t)t * c->d_s + j];
                    z[j] = acc;
                }
                build_lut(z, c->C, c->M, dsub, lut);
            }
            for (int64_t p2 = c->off[l]; p2 < c->off[l + 1]; ++p2) {
                int64_t id = c->ids[p2];
                const uint8_t *code = c->codes + id * c->M;
                double acc = 0.0;
                for (int m = 0; m < c->M; ++m) acc += lut[m * 256 + code[m]];
                cs[w].dist = acc;
                cs[w].id = id;
                ++w;
            }
        }
        qsort(cs, (size_t)w, sizeof(cand), cand_cmp);
        int64_t nres = w;
        if (c->rerank_k > 0) {
            nres = w < c->rerank_k ? w : c->rerank_k;
            for (int64_t r = 0; r < nres; ++r)
                cs[r].dist = scan_dist(qs, c->db + cs[r].id * c->d, c->d_s, c->normalize, xbuf);
            qsort(cs, (size_t)nres, sizeof(cand), cand_cmp);
        }
        for (int r = 0; r < c->k_out; ++r) {
            if (r < nres) {
                c->out_ids[qi * c->k_out + r] = cs[r].id;
                c->out_dist[qi * c->k_out + r] = cs[r].dist;
            } else {
                c->out_ids[qi * c->k_out + r] = -1;
                c->out_dist[qi * c->k_out + r] = INFINITY;
            }
        }
        free(cs);
    }
    free(qbuf); free(qs); free(z); free(xbuf); free(lut); free(cbuf); free(probes);
}

int orc_ivfopq_search(const float *db, int64_t N, int d, const float *cent, int nlist, int ldc,
                      const int64_t *list_off, const int32_t *list_ids, const float *R,
                      const float *codebooks, const uint8_t *codes, int M,
                      const float *queries, int64_t B, int d_c, int d_s, int nprobe, int k_out,
                      int rerank_k, int normalize, const float *lcent, int64_t *out_ids,
                      double *out_dist, int32_t *out_probes, double *out_pdist, int nthreads) {
    (void)N;
    if (d_c < 1 || d_c > ldc || d_s < 1 || d_s > d || nprobe < 1 || nprobe > nlist ||
        k_out < 1 || M < 1 || d_s % M != 0 || rerank_k < 0)
        return -1;
    opq_ctx c = {db, d, cent, nlist, ldc, list_off, list_ids, R, codebooks, codes, M, queries,
                 d_c, d_s, nprobe, k_out, rerank_k, normalize, out_ids, out_dist, out_probes,
                 out_pdist, nprobe + 1, lcent};
    parallel_for(B, nthreads, opq_range, &c);
    return 0;
}
