/*
 * FP64 CPU oracle for the low-dimensional graph shortlist of AdANNS-DiskANN
 * (test infrastructure only; shares no code with the GPU library).
 *
 * Sec. 4.3 "AdANNS for Composite Indices" and the AdANNS-DiskANN appendix:
 * the search graph is formed with a low-d MR and its shortlist is re-ranked
 * with a high-d MR.  The graph here is a DiskANN-style pruned proximity graph
 * built in one pass, written from the method's definition:
 *   1. candidates: the K nearest other rows of every row at dimension m;
 *   2. robust prune of each candidate list with factor alpha to at most R
 *      out-neighbours (take the nearest remaining candidate c, drop every
 *      remaining v with alpha * d(c, v) <= d(p, v));
 *   3. every edge p -> c also offers p to c; a row whose own and offered
 *      neighbours exceed R is pruned again over their union;
 *   4. entry point: the row nearest to the mean of all rows.
 * The search is best-first with a bounded candidate list of L entries:
 * repeatedly expand the nearest not-yet-expanded entry, offer its
 * neighbours that are not in the list, keep the L nearest by (distance, id),
 * until every entry is expanded.
 *
 * Rows are given already at dimension m (prefix-normalised by the caller when
 * the metric asks for it); distances are squared L2 in FP64.  Ties are broken
 * by the smaller id.  Decisions whose two distances lie within the caller's
 * tolerance are reported as ambiguous per row / per query, so a comparison
 * with an FP32 implementation can skip them.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef void (*g_range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct { g_range_fn fn; void *ctx; int64_t lo, hi; } g_job;

static void *g_run(void *p) {
    g_job *j = (g_job *)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void g_parallel(int64_t n, int nthreads, g_range_fn fn, void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > n) nthreads = (int)(n > 0 ? n : 1);
    pthread_t th[256];
    g_job jobs[256];
    int64_t per = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].lo = t * per < n ? t * per : n;
        jobs[t].hi = (t + 1) * per < n ? (t + 1) * per : n;
        pthread_create(&th[t], NULL, g_run, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

static double sqd(const double *a, const double *b, int m) {
    double acc = 0.0;
    for (int j = 0; j < m; ++j) {
        double d = a[j] - b[j];
        acc += d * d;
    }
    return acc;
}

static int near_equal(double a, double b, double rel, double abs_) {
    double hi = a > b ? a : b;
    return fabs(a - b) <= rel * fabs(hi) + abs_;
}

typedef struct { double d; int64_t id; } gkey;

static int gkey_cmp(const void *pa, const void *pb) {
    const gkey *a = (const gkey *)pa, *b = (const gkey *)pb;
    if (a->d < b->d) return -1;
    if (a->d > b->d) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

static int gkey_less(gkey a, gkey b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

/* ------------------------------------------------------------------ */
/* 1. K nearest other rows                                             */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *X; int64_t N; int m, K; double rel, abs_;
    int32_t *nbr; double *dist; uint8_t *amb;
} knn_ctx;

static void knn_range(void *p, int64_t lo, int64_t hi) {
    knn_ctx *c = (knn_ctx *)p;
    gkey *all = (gkey *)malloc(sizeof(gkey) * (size_t)c->N);
    for (int64_t i = lo; i < hi; ++i) {
        int64_t w = 0;
        for (int64_t j = 0; j < c->N; ++j) {
            if (j == i) continue;
            all[w].d = sqd(c->X + i * c->m, c->X + j * c->m, c->m);
            all[w].id = j;
            ++w;
        }
        qsort(all, (size_t)w, sizeof(gkey), gkey_cmp);
        int K = c->K < w ? c->K : (int)w;
        for (int r = 0; r < c->K; ++r) {
            c->nbr[i * c->K + r] = r < K ? (int32_t)all[r].id : -1;
            c->dist[i * c->K + r] = r < K ? all[r].d : INFINITY;
        }
        c->amb[i] = (uint8_t)(K < w && near_equal(all[K - 1].d, all[K].d, c->rel, c->abs_));
    }
    free(all);
}

int orc_knn_graph(const double *X, int64_t N, int m, int K, double rel, double abs_, int32_t *nbr,
                  double *dist, uint8_t *amb, int nthreads) {
    if (N < 2 || m < 1 || K < 1) return -1;
    knn_ctx c = {X, N, m, K, rel, abs_, nbr, dist, amb};
    g_parallel(N, nthreads, knn_range, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 2. robust prune of one row's candidates (sorted by (distance, id))  */
/* ------------------------------------------------------------------ */
static int robust_prune(const double *X, int m, int64_t p, gkey *cand, int nc, double alpha,
                        int R, int32_t *out, double rel, double abs_, uint8_t *amb) {
    int nout = 0;
    char *alive = (char *)malloc((size_t)(nc > 0 ? nc : 1));
    for (int i = 0; i < nc; ++i) alive[i] = cand[i].id != p;
    for (int i = 0; i < nc && nout < R; ++i) {
        if (!alive[i]) continue;
        int64_t c = cand[i].id;
        out[nout++] = (int32_t)c;
        alive[i] = 0;
        for (int j = i + 1; j < nc; ++j) {
            if (!alive[j]) continue;
            double dcv = alpha * sqd(X + c * m, X + cand[j].id * m, m);
            if (near_equal(dcv, cand[j].d, rel, abs_)) *amb = 1;
            if (dcv <= cand[j].d) alive[j] = 0;
        }
    }
    free(alive);
    return nout;
}

typedef struct {
    const double *X; int m, K, R; double alpha, rel, abs_;
    const int32_t *knn; const double *kd; int32_t *out; int32_t *nout; uint8_t *amb;
} prune_ctx;

static void prune_range(void *p, int64_t lo, int64_t hi) {
    prune_ctx *c = (prune_ctx *)p;
    gkey *cand = (gkey *)malloc(sizeof(gkey) * (size_t)c->K);
    for (int64_t i = lo; i < hi; ++i) {
        int nc = 0;
        for (int r = 0; r < c->K; ++r)
            if (c->knn[i * c->K + r] >= 0) {
                cand[nc].id = c->knn[i * c->K + r];
                cand[nc].d = c->kd[i * c->K + r];
                ++nc;
            }
        c->nout[i] = robust_prune(c->X, c->m, i, cand, nc, c->alpha, c->R, c->out + i * c->R,
                                  c->rel, c->abs_, c->amb + i);
    }
    free(cand);
}

/* ------------------------------------------------------------------ */
/* 3. offered (reverse) edges and the final pruning                     */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *X; int m, R; double alpha, rel, abs_;
    const int32_t *fwd; const int32_t *nfwd;
    const int64_t *roff; const int32_t *rev;
    int32_t *graph; uint8_t *amb;
} final_ctx;

static void final_range(void *p, int64_t lo, int64_t hi) {
    final_ctx *c = (final_ctx *)p;
    for (int64_t q = lo; q < hi; ++q) {
        int64_t nr = c->roff[q + 1] - c->roff[q];
        int cap = c->nfwd[q] + (int)nr;
        gkey *u = (gkey *)malloc(sizeof(gkey) * (size_t)(cap > 0 ? cap : 1));
        int nu = 0;
        for (int r = 0; r < c->nfwd[q]; ++r) u[nu++].id = c->fwd[q * c->R + r];
        for (int64_t r = 0; r < nr; ++r) u[nu++].id = c->rev[c->roff[q] + r];
        for (int i = 0; i < nu; ++i) u[i].d = sqd(c->X + q * c->m, c->X + u[i].id * c->m, c->m);
        qsort(u, (size_t)nu, sizeof(gkey), gkey_cmp);
        int w = 0;  /* drop duplicates (same id, adjacent after the sort) */
        for (int i = 0; i < nu; ++i)
            if (w == 0 || u[i].id != u[w - 1].id || u[i].d != u[w - 1].d) u[w++] = u[i];
        nu = w;
        int32_t *row = c->graph + q * c->R;
        int nout;
        if (nu <= c->R) {
            for (int i = 0; i < nu; ++i) row[i] = (int32_t)u[i].id;
            nout = nu;
        } else {
            nout = robust_prune(c->X, c->m, q, u, nu, c->alpha, c->R, row, c->rel, c->abs_,
                                c->amb + q);
        }
        for (int i = nout; i < c->R; ++i) row[i] = -1;
        free(u);
    }
}

/* The whole build.  graph: N x R ids (-1 padding), each row sorted by
 * (distance, id).  amb[p] = 1 when a decision for row p was within the
 * tolerance.  *entry = the row nearest to the mean row (ties: smaller id). */
int orc_graph_build(const double *X, int64_t N, int m, int K, int R, double alpha, double rel,
                    double abs_, int32_t *graph, uint8_t *amb, int64_t *entry, int nthreads) {
    if (N < 2 || m < 1 || K < 1 || R < 1 || !(alpha >= 1.0)) return -1;
    int32_t *knn = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * K);
    double *kd = (double *)malloc(sizeof(double) * (size_t)N * K);
    int32_t *fwd = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * R);
    int32_t *nfwd = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t *roff = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    memset(amb, 0, (size_t)N);
    orc_knn_graph(X, N, m, K, rel, abs_, knn, kd, amb, nthreads);
    prune_ctx pc = {X, m, K, R, alpha, rel, abs_, knn, kd, fwd, nfwd, amb};
    g_parallel(N, nthreads, prune_range, &pc);
    /* offered edges, grouped by target in ascending source order */
    for (int64_t p = 0; p < N; ++p)
        for (int r = 0; r < nfwd[p]; ++r) roff[fwd[p * R + r] + 1] += 1;
    for (int64_t q = 0; q < N; ++q) roff[q + 1] += roff[q];
    int32_t *rev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(roff[N] > 0 ? roff[N] : 1));
    int64_t *fill = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    for (int64_t p = 0; p < N; ++p)
        for (int r = 0; r < nfwd[p]; ++r) {
            int32_t q = fwd[p * R + r];
            rev[roff[q] + fill[q]++] = (int32_t)p;
        }
    final_ctx fc = {X, m, R, alpha, rel, abs_, fwd, nfwd, roff, rev, graph, amb};
    g_parallel(N, nthreads, final_range, &fc);
    /* entry point */
    double *mean = (double *)calloc((size_t)m, sizeof(double));
    for (int64_t p = 0; p < N; ++p)
        for (int j = 0; j < m; ++j) mean[j] += X[p * m + j];
    for (int j = 0; j < m; ++j) mean[j] /= (double)N;
    gkey best = {INFINITY, -1};
    for (int64_t p = 0; p < N; ++p) {
        gkey k = {sqd(X + p * m, mean, m), p};
        if (gkey_less(k, best)) best = k;
    }
    *entry = best.id;
    free(mean); free(fill); free(rev); free(roff); free(nfwd); free(fwd); free(kd); free(knn);
    return 0;
}

/* ------------------------------------------------------------------ */
/* best-first search with a bounded candidate list                      */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *X; int64_t N; int m; const int32_t *graph; int R; int64_t entry;
    const double *Q; int L, kk; double rel, abs_;
    int64_t *out_ids; double *out_dist; uint8_t *amb; int64_t *nexp;
} gs_ctx;

static void gs_range(void *p, int64_t lo, int64_t hi) {
    gs_ctx *c = (gs_ctx *)p;
    gkey *lst = (gkey *)malloc(sizeof(gkey) * (size_t)(c->L + c->R + 1));
    char *done = (char *)malloc((size_t)(c->L + c->R + 1));
    for (int64_t qi = lo; qi < hi; ++qi) {
        const double *q = c->Q + qi * c->m;
        int n = 1;
        uint8_t amb = 0;
        int64_t nexp = 0;
        lst[0].id = c->entry;
        lst[0].d = sqd(q, c->X + c->entry * c->m, c->m);
        done[0] = 0;
        for (;;) {
            /* the nearest entry not yet expanded (the list is kept sorted) */
            int sel = -1, sel2 = -1;
            for (int i = 0; i < n; ++i)
                if (!done[i]) {
                    if (sel < 0) sel = i;
                    else { sel2 = i; break; }
                }
            if (sel < 0) break;
            if (sel2 >= 0 && near_equal(lst[sel].d, lst[sel2].d, c->rel, c->abs_)) amb = 1;
            done[sel] = 1;
            ++nexp;
            int64_t v = lst[sel].id;
            /* offer its neighbours that are not in the list */
            for (int r = 0; r < c->R; ++r) {
                int64_t u = c->graph[v * c->R + r];
                if (u < 0) continue;
                int in = 0;
                for (int i = 0; i < n; ++i)
                    if (lst[i].id == u) { in = 1; break; }
                if (in) continue;
                gkey k = {sqd(q, c->X + u * c->m, c->m), u};
                if (n == c->L) {
                    if (near_equal(k.d, lst[n - 1].d, c->rel, c->abs_)) amb = 1;
                    if (!gkey_less(k, lst[n - 1])) continue;
                    --n;  /* the current worst leaves */
                }
                int pos = n;
                while (pos > 0 && gkey_less(k, lst[pos - 1])) {
                    lst[pos] = lst[pos - 1];
                    done[pos] = done[pos - 1];
                    --pos;
                }
                lst[pos] = k;
                done[pos] = 0;
                ++n;
            }
        }
        if (c->kk < n && near_equal(lst[c->kk - 1].d, lst[c->kk].d, c->rel, c->abs_)) amb = 1;
        for (int r = 0; r < c->kk; ++r) {
            c->out_ids[qi * c->kk + r] = r < n ? lst[r].id : -1;
            c->out_dist[qi * c->kk + r] = r < n ? lst[r].d : INFINITY;
        }
        c->amb[qi] = amb;
        c->nexp[qi] = nexp;
    }
    free(lst);
    free(done);
}

int orc_graph_search(const double *X, int64_t N, int m, const int32_t *graph, int R,
                     int64_t entry, const double *Q, int64_t B, int L, int kk, double rel,
                     double abs_, int64_t *out_ids, double *out_dist, uint8_t *amb,
                     int64_t *nexp, int nthreads) {
    if (N < 1 || m < 1 || R < 1 || L < 1 || kk < 1 || kk > L || entry < 0 || entry >= N)
        return -1;
    gs_ctx c = {X, N, m, graph, R, entry, Q, L, kk, rel, abs_, out_ids, out_dist, amb, nexp};
    g_parallel(B, nthreads, gs_range, &c);
    return 0;
}
