/*
 * adanns.h -- C ABI of the GB300 (sm_103a) AdANNS search library.
 *
 * AdANNS-IVF (Sec. 4.1, Algorithm 1, Table "formula" AdANNS-IVF row): queries
 * are mapped to k-means centroids with the first d_c coordinates of a nested
 * (Matryoshka) embedding, the n_p nearest inverted lists are scanned with the
 * first d_s coordinates, and a fused top-k returns ids and distances.
 *
 * Conventions shared by every entry point
 *  - All array arguments are DEVICE pointers into memory the caller owns,
 *    unless a parameter says otherwise.  Row-major, densely packed, FP32
 *    unless stated.  Every call is asynchronous on `cuda_stream` (a
 *    cudaStream_t; NULL = the legacy default stream) unless it says it
 *    synchronises.  Outputs are valid once the stream reaches the call.
 *  - Distances are squared L2.  With ADANNS_METRIC_L2_PREFIXNORM an m-prefix
 *    used as a representation is L2-normalised at its own length,
 *    P_m(v) = v[0:m] / ||v[0:m]||, P_m(0) = 0 (Sec. 3 "Matryoshka
 *    Representations": the first m coordinates form an m-dim representation),
 *    and dist_m(q, x) = ||P_m(q) - P_m(x)||^2.  ADANNS_METRIC_L2 uses raw
 *    prefixes.
 *  - Ties among equal distances are ordered by ascending database id (list
 *    id for the cluster mapping).  Fewer than k candidates are padded with
 *    id -1 and distance +inf.
 *  - Return value: ADANNS_OK (0) or a negative ADANNS_ERR_* code; the message
 *    is available from adanns_last_error() on the calling thread.  No entry
 *    point aborts or traps.  Input values must be finite.
 *  - Prefix lengths (d_c, d_s) must belong to the MR granularity set
 *    G = {8,16,32,48,64,96,128,192,256,384,512,768,1024,2048} and not exceed
 *    the stored dimension (the paper's nested sizes, Sec. 3 "Encoders").
 */
#ifndef ADANNS_H
#define ADANNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADANNS_OK 0
#define ADANNS_ERR_ARG (-1)     /* invalid argument (null pointer, size out of range) */
#define ADANNS_ERR_DIM (-2)     /* prefix length not in G, or beyond the index */
#define ADANNS_ERR_OOM (-3)     /* device allocation failed */
#define ADANNS_ERR_CUDA (-4)    /* a CUDA runtime call or launch failed */
#define ADANNS_ERR_TIMEOUT (-5) /* a bounded device wait gave up */
#define ADANNS_ERR_STATE (-6)   /* the index lacks the requested storage / OPQ data */

#define ADANNS_METRIC_L2 0
#define ADANNS_METRIC_L2_PREFIXNORM 1

/* storage tiers of the database vectors (bit mask for builders; one value for
 * search).  F32 is always kept (the exact scan and the rerank read it).  BF16
 * and FP8-E4M3 copies store x / s_x per vector with s_x = max_j |x_j| / R
 * (R = 1 for BF16, 448 for FP8-E4M3) in the same prefix-major list layout. */
#define ADANNS_STORE_F32 1
#define ADANNS_STORE_BF16 2
#define ADANNS_STORE_FP8E4M3 4

typedef struct adanns_index adanns_index; /* opaque; device memory owned by the library */

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next call on the same thread. */
const char *adanns_last_error(void);

/* ABI version of this header (major * 100 + minor). */
int adanns_version(void);

/* Number of CUDA kernels this library has launched since it was loaded, on
 * all threads (a diagnostic counter; host-side, no device access). */
int64_t adanns_launch_count(void);

/*
 * Runtime options (process-wide, every device; host-side, no device access).
 * They select among kernels that compute the same result, bound scratch and
 * waits, and hold test hooks.  The first call of any entry point seeds the
 * first five from the environment variables ADANNS_FP32_STREAM,
 * ADANNS_ADC_SELECT, ADANNS_COARSE_TC, ADANNS_RERANK_PRUNE ("0" turns the
 * feature off) and ADANNS_SCRATCH_GB (GiB); nothing reads the environment
 * after that.  A change applies to calls issued after it; a search plan keeps
 * what it captured.
 *   ADANNS_OPT_FP32_STREAM    1 (default): streaming FP32 scan where few
 *                             queries share a probed list; 0: tiled scan always
 *   ADANNS_OPT_ADC_SELECT     1 (default): IVF-OPQ distance-then-select stage
 *                             for nprobe <= 256; 0: running top-k per list
 *   ADANNS_OPT_COARSE_TC      1 (default): tensor-core cluster mapping where it
 *                             applies; 0: FP32 kernels only
 *   ADANNS_OPT_RERANK_PRUNE   1 (default): certified pruning of the shortlist
 *                             before the exact rerank; 0: rerank all of it
 *   ADANNS_OPT_SCRATCH_BYTES  scratch one search call may hold (default
 *                             12 GiB, at least 1 MiB); larger batches are sliced
 *   ADANNS_OPT_WAIT_LIMIT_NS  bound of every tensor-core pipeline wait
 *                             (default 2e9 ns, within [1e5, 6e10]); a wait that
 *                             runs out is reported by adanns_index_status
 *   ADANNS_OPT_SCAN_FILTER    0 (default): every approximate distance of the
 *                             BF16 / FP8 tensor-core scan is written (2 bytes)
 *                             and the shortlist selected afterwards; 1: each
 *                             query's nearest list is scanned first and, in the
 *                             other lists, only members whose approximate
 *                             distance can still enter the shortlist leave the
 *                             SM (as 4-byte records).  Both give the same
 *                             result.  Lists of more than 65,536 members always
 *                             take the first.
 *   ADANNS_OPT_NARROW_SCAN    1 (default): when few queries share a probed
 *                             list (at most 24 on average) and the prefix spans
 *                             16 or more K-blocks (d_s >= 1024 for BF16, 2048
 *                             for FP8), the BF16 / FP8 tensor-core scan takes
 *                             tiles of 128 members x 32 queries instead of 128
 *                             queries x 256 members; 2: those tiles at any d_s
 *                             when few queries share a list; 0: the wide tiles
 *                             always.  The approximate keys agree (the tensor
 *                             cores may round the dot products of the two tile
 *                             shapes differently in the last FP32 place); the
 *                             exact rerank follows.
 *   ADANNS_OPT_TEST_SKIP_LOAD test hook, -1 (default).  n >= 0 makes the next
 *                             tensor-core scan launch (one launch; the option
 *                             then returns to -1) leave out stage load n (in
 *                             member-tile, K-block order) of its work item 0 --
 *                             no copy and no arrival -- so that the MMA
 *                             issuer's bounded wait runs out and the timeout
 *                             path runs (nothing happens when item 0 has fewer
 *                             loads).  That call's results are invalid.  Never
 *                             needed outside tests.
 * adanns_set_option returns ADANNS_ERR_ARG for an unknown option or a value
 * out of range (the option keeps its value).
 */
#define ADANNS_OPT_FP32_STREAM 0
#define ADANNS_OPT_ADC_SELECT 1
#define ADANNS_OPT_COARSE_TC 2
#define ADANNS_OPT_RERANK_PRUNE 3
#define ADANNS_OPT_SCRATCH_BYTES 4
#define ADANNS_OPT_WAIT_LIMIT_NS 5
#define ADANNS_OPT_TEST_SKIP_LOAD 6
#define ADANNS_OPT_SCAN_FILTER 7
#define ADANNS_OPT_NARROW_SCAN 8
#define ADANNS_OPT_COUNT 9
int adanns_set_option(int option, int64_t value);
int adanns_get_option(int option, int64_t *value);

/*
 * Stage timing (diagnostics).  adanns_profile_enable(1) starts recording a
 * CUDA event pair, on the call's stream, around each stage of every search
 * (0 query prep, 1 cluster mapping, 2 probe inversion, 3 list scan, 4 merge,
 * further ids for later stages); enabling or disabling discards the records.
 * adanns_profile_read synchronises on the recorded events and fills host
 * arrays ms[s] (summed milliseconds) and count[s] (records) for s < nstage.
 */
int adanns_profile_enable(int on);
int adanns_profile_read(double *ms, int64_t *count, int nstage);
/* Host wall time (microseconds, summed) spent issuing each stage's work. */
int adanns_profile_read_host(double *us, int nstage);
/*
 * Work counters summed over the calls made while profiling was on (the
 * device values are read after a device synchronisation):
 *   values[0]  (query, candidate) pairs re-scored by the exact rerank of the
 *              low-precision tiers, after the certified pruning
 *   values[1]  shortlist slots (queries x rerank_k) of those calls
 *   values[2]  candidates kept for the exact shortlist selection: by the
 *              filtered tensor-core scan (ADANNS_OPT_SCAN_FILTER), else by
 *              the selection's own threshold pass over the scan's keys
 *   values[3]  queries whose kept candidates missed the selection's
 *              on-chip buffer (too many, or fewer than the shortlist), so
 *              that they were selected from global memory instead
 * Entries beyond the known counters are 0.
 */
int adanns_profile_read_counters(int64_t *values, int ncounter);

/*
 * Build an AdANNS-IVF index (Algorithm 1 adannsConstruction; Sec. 3 "IVF":
 * Lloyd k-means coarse quantiser and inverted lists, clustering on the d_c
 * prefix as in Sec. 4.1).
 *   db        N x d FP32, device, caller-owned; copied (re-laid out) into the
 *             index, so it may be freed after the call returns.
 *   d_c       clustering prefix (in G, <= d); nlist clusters, 1 <= nlist <= train_n.
 *   niter     Lloyd iterations (>= 0).
 *   train_n   training sample size, nlist <= train_n <= N.  The sample is the
 *             first train_n entries of a splitmix64(seed) Fisher-Yates shuffle
 *             of [0, N); the initial centroids are the sample rows at the first
 *             nlist entries of a splitmix64(seed + 1) shuffle of [0, train_n).
 *   metric    ADANNS_METRIC_*; storage_mask must include ADANNS_STORE_F32.
 *   objective optional HOST pointer to niter doubles: the k-means objective
 *             (sum of squared distances) at each iteration's assignment.
 * Ties in the assignment go to the smallest cluster index; an empty cluster
 * keeps its previous centroid.  Centroid sums are accumulated in FP64.
 * Synchronises `cuda_stream` (the objective is read back every iteration).
 * On success *out owns the index; release it with adanns_index_free.
 */
int adanns_build_ivf(const float *db, int64_t N, int d, int d_c, int nlist, int niter,
                     int64_t train_n, uint64_t seed, int metric, int storage_mask,
                     double *objective, void *cuda_stream, adanns_index **out);

/*
 * Create an index from given centroids and list assignment (import path; the
 * same layout adanns_build_ivf produces).
 *   db         N x d FP32 (device), centroids nlist x d_c FP32 (device),
 *   assign     N int32 in [0, nlist) (device).
 * Members of each list are ordered by ascending id.  Synchronises the stream.
 * With nlist = 1 (one list holding every row) a search with nprobe = 1 is
 * exhaustive: adanns_search_ivfopq is then the exhaustive AdANNS-OPQ search of
 * Sec. 4.2 (ADC over every code) and adanns_search_ivf brute force at d_s.
 */
int adanns_index_create(const float *db, int64_t N, int d, const float *centroids, int nlist,
                        int d_c, const int32_t *assign, int metric, int storage_mask,
                        void *cuda_stream, adanns_index **out);

/* Sizes of an index (any pointer may be NULL). Host outputs. */
int adanns_index_info(const adanns_index *idx, int64_t *N, int *d, int *d_c, int *nlist,
                      int *metric);

/* OPQ shape of an index (host outputs, either may be NULL): the prefix d_s
 * and the code bytes M, both 0 when the index holds no OPQ data. */
int adanns_index_opq_info(const adanns_index *idx, int *d_s, int *M);

/* Copy the CSR lists to device buffers: list_off int64 [nlist + 1] (member
 * offsets), list_ids int32 [N] (database ids, ascending inside each list). */
int adanns_index_get_lists(const adanns_index *idx, int64_t *list_off, int32_t *list_ids,
                           void *cuda_stream);

/* Copy the FP32 centroids (nlist x d_c) to a device buffer. */
int adanns_index_get_centroids(const adanns_index *idx, float *centroids, void *cuda_stream);

/* Status of the index's device work: synchronises the stream, returns
 * ADANNS_ERR_TIMEOUT if a bounded wait of a tensor-core pipeline gave up since
 * the last check (the results of that call are then invalid), and clears it. */
int adanns_index_status(const adanns_index *idx, void *cuda_stream);

/* Upper bound of the scratch bytes adanns_search_ivf holds at once for these
 * arguments (host-side arithmetic, no device access); -1 for bad arguments.
 * Used for admission by device memory. */
int64_t adanns_search_scratch_bytes(const adanns_index *idx, int64_t B, int d_c, int d_s,
                                    int nprobe, int k, int storage, int rerank_k);

/* Release an index (NULL is ignored).  Waits for the device to finish using it. */
void adanns_index_free(adanns_index *idx);

/*
 * Index files.  The index is formed once and then serves many queries (Sec. 5
 * "Search for AdANNS Hyperparameters"), so it can be written to a file and
 * loaded by another process instead of being rebuilt.
 *
 * adanns_index_export writes to the HOST path `path` (created or truncated)
 * what defines the index: a 96-byte header (magic "ADANNSIX", format version
 * 1, N, d, d_c, nlist, metric, storage mask, OPQ d_s and M, OPQ flags with
 * bit 0 = residual codes), the FP32 centroids [nlist][d_c], the list of every
 * database id (int32 [N]), the database rows in id order (FP32 [N][d],
 * recovered from the index's own copy), with OPQ data the rotation
 * [d_s][d_s], the codebooks [M][256][d_s / M] and the codes in id order
 * (uint8 [N][M]), and with residual codes the list centres [nlist][d_s]; all
 * little-endian, packed.  It synchronises the stream.  The file is about as
 * large as the database.  Errors: ADANNS_ERR_ARG (NULL argument, the file
 * cannot be opened or written).
 *
 * adanns_index_import reads such a file and builds the index with
 * adanns_index_create (the same storage tiers) and, when present,
 * adanns_index_set_opq, so the imported index searches exactly like the
 * exported one.  It allocates the database rows on the device for the
 * duration of the call, synchronises the stream, and on success *out owns the
 * index (release with adanns_index_free).  Errors: ADANNS_ERR_ARG (NULL
 * argument, file cannot be opened), ADANNS_ERR_STATE (not an index file, other
 * version, inconsistent sizes, truncated or over-long file), plus those of
 * adanns_index_create.
 */
int adanns_index_export(const adanns_index *idx, const char *path, void *cuda_stream);
int adanns_index_import(const char *path, void *cuda_stream, adanns_index **out);

/*
 * Lloyd assignment step (Sec. 3 "IVF"): for each of n points (rows of `ld`
 * floats, first `dim` used, prefix-normalised at dim under
 * ADANNS_METRIC_L2_PREFIXNORM) the nearest of nc centroids (nc x dim FP32),
 * ties to the smallest index.  out_assign int32 [n]; out_dist FP32 [n]
 * (squared distance, may be NULL).  dim in G, 1 <= nc.
 */
int adanns_kmeans_assign(const float *points, int64_t n, int ld, int dim, int metric,
                         const float *centroids, int nc, int32_t *out_assign, float *out_dist,
                         void *cuda_stream);

/*
 * Lloyd update step (Sec. 3 "IVF"): centroid h becomes the mean of the
 * (normalised, as above) points assigned to it, summed in FP64 and rounded
 * to FP32; a cluster with no point keeps its value.  centroids is read and
 * overwritten (nc x dim FP32).
 */
int adanns_kmeans_update(const float *points, int64_t n, int ld, int dim, int metric,
                         const int32_t *assign, int nc, float *centroids, void *cuda_stream);

/*
 * AdANNS-IVF search (Algorithm 1 adannsInference; Table "formula"
 * AdANNS-IVF row):
 *   h(q): the nprobe nearest centroids to P_dc(q) by (distance, list id);
 *   result: the k nearest members of those lists to q by dist_ds, then id.
 *   queries  B x d FP32 (device); d_c in G and <= the index's d_c; d_s in G,
 *            d_s <= d; 1 <= nprobe <= nlist; 1 <= k <= 1024.
 *            A d_c below the built one is AdANNS-IVF-D (Table "formula"
 *            IVF-D row; Sec. 5.1): the lists built at the larger prefix are
 *            probed with P_dc(q) against the first d_c coordinates of each
 *            centroid, taken as stored (not renormalised).
 *   storage  ADANNS_STORE_F32: the exact FP32 scan (rerank_k must be 0).
 *            With few queries per probed list (B * nprobe / nlist <= 16,
 *            nprobe <= 256) the lists are streamed once per 16-query tile
 *            and the distances selected per query afterwards (4 bytes per
 *            probed member of scratch); ADANNS_FP32_STREAM=0 keeps the
 *            shared-memory tiled scan.  Both give the same result.
 *            ADANNS_STORE_BF16 / ADANNS_STORE_FP8E4M3 (tier built into the
 *            index, metric ADANNS_METRIC_L2_PREFIXNORM, nprobe <= 128): the
 *            probed lists are scanned on the tensor cores with FP32
 *            accumulation, giving approximate distances
 *            |P(q)|^2 + |P(x)|^2 - 2 s_q s_x nu_x (q_low . x_low); the
 *            rerank_k (k <= rerank_k <= 2048) best of those are re-scored
 *            with the exact FP32 dist_ds (Sec. 4.3 shortlist-rerank) and the
 *            k best by (distance, id) are returned -- the returned distances
 *            are exact; ids can differ from the FP32 scan where the exact
 *            top-k was not in the approximate shortlist.  A tensor-core
 *            pipeline timeout is reported by adanns_index_status.
 *   out_ids  int64 [B x k], out_dist FP32 [B x k] (device, caller-owned).
 *   out_probes optional int32 [B x nprobe]: the probed lists, nearest first.
 * Scratch memory is taken from the CUDA stream-ordered allocator and returned
 * before the call's work completes; B is processed in slices so scratch
 * stays bounded (about 2 GiB).
 */
int adanns_search_ivf(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                      int d_s, int nprobe, int k, int storage, int rerank_k, int64_t *out_ids,
                      float *out_dist, int32_t *out_probes, void *cuda_stream);

/* AdANNS-IVF search of HOST queries with HOST results: adanns_search_ivf's
 * arguments and rules, but queries (B x d FP32), out_ids (int64 B x k) and
 * out_dist (FP32 B x k) are host memory.
 *   slice 0 and all three buffers page-locked (cudaHostAlloc, or registered):
 *            the GPU reads the queries in place (only the first
 *            max(d_c, d_s) coordinates of each row cross the host link) and
 *            writes the results in place; no copy, the batch stays whole.
 *   otherwise: the batch is cut into slices of `slice` rows (0: four slices);
 *            slice i+1's queries are copied to the device on an internal
 *            stream while slice i is searched on cuda_stream, and slice i's
 *            results are copied back while slice i+1 is searched (the copies
 *            of pageable buffers run synchronously).
 * Returns once the work is queued; the results are on the host when
 * cuda_stream reaches the point of the call (synchronise it, or an event
 * recorded after the call).  The host buffers must stay valid until then.
 * Results equal adanns_search_ivf on the same rows. */
int adanns_search_ivf_host(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                           int d_s, int nprobe, int k, int storage, int rerank_k,
                           int64_t *out_ids, float *out_dist, int64_t slice, void *cuda_stream);

/* AdANNS-IVF search of a batch whose queries carry their own budgets (Sec. 5
 * "Compute-aware Elastic Search During Inference": each query picks its
 * d_s, nprobe and k at run time over one resident index), in one pass of the
 * search's kernels instead of one call per budget.
 *   d_s, nprobe, k  HOST int32 arrays of B entries, read before the call
 *            returns: query i is searched with d_s[i], nprobe[i], k[i] under
 *            the rules of adanns_search_ivf, and k[i] <= k_max <= 1024.
 *   storage  ADANNS_STORE_F32 (rerank_k 0, nprobe[i] <= 256): the streaming
 *            FP32 scan, every query at its own d_s.  ADANNS_STORE_BF16 /
 *            ADANNS_STORE_FP8E4M3: every d_s[i] must be equal (the
 *            tensor-core scan tiles share one K extent) and
 *            k_max <= rerank_k <= 2048, nprobe[i] <= 128; the shortlist is
 *            the rerank_k best of each query's own probed lists.
 *   out_ids  int64 [B x k_max], out_dist FP32 [B x k_max] (device): row i
 *            holds query i's k[i] results, then (-1, +inf) up to k_max.
 * Row i equals the first k[i] entries of adanns_search_ivf on query i alone
 * with (d_c, d_s[i], nprobe[i], k_max, storage, rerank_k): for the FP32 tier
 * that is its exact top-k[i]; for the low-precision tiers the top-k[i] of the
 * re-scored shortlist.  ADANNS_ERR_ARG / ADANNS_ERR_DIM for a bad entry (its
 * index in the message); nothing is launched then.
 */
int adanns_search_ivf_budgets(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                              const int32_t *d_s, const int32_t *nprobe, const int32_t *k,
                              int k_max, int storage, int rerank_k, int64_t *out_ids,
                              float *out_dist, void *cuda_stream);

/* ------------------------------------------------------------------------
 * AdANNS-OPQ on the d_s prefix and the AdANNS-IVFOPQ composite
 * (Sec. 3 "OPQ": M sub-vectors, 2^8 codewords each, m bytes per vector,
 * search by M codebook lookups, an orthonormal rotation R learned first;
 * Sec. 4.2: OPQ on the first d_s coordinates of the MR, sub-vectors of
 * d_s / M dimensions; Sec. 4.3 and Table "formula" IVFOPQ row: IVF at d_c
 * with OPQ distances inside the probed lists, read as asymmetric lookup).
 * Layouts: R is d_s x d_s row-major with z = x R (x a row vector);
 * codebooks are M x 256 x (d_s / M) FP32; codes are N x M bytes.
 * The vector quantised is z = P_ds(x) R (the prefix normalised under
 * ADANNS_METRIC_L2_PREFIXNORM, raw under ADANNS_METRIC_L2).  d_s must be in G,
 * M must divide d_s, d_s / M <= 64.
 * ---------------------------------------------------------------------- */

/* Encode n rows (ld floats each; first d_s used): codes[i][m] = the nearest
 * codeword of subspace m to z_i (squared L2, ties to the smallest codeword). */
int adanns_opq_encode(const float *x, int64_t n, int ld, int d_s, int M, int metric,
                      const float *R, const float *codebooks, uint8_t *codes, void *cuda_stream);

/* One PQ Lloyd update: codeword (m, c) becomes the FP64 mean of the
 * subspace-m slices of the rows of z (n x d_s, already rotated) whose code is
 * c, rounded to FP32; a codeword with no member keeps its value. */
int adanns_pq_update(const float *z, int64_t n, int d_s, int M, const uint8_t *codes,
                     float *codebooks, void *cuda_stream);

/* Orthogonal Procrustes step of OPQ: R = argmin over orthogonal R of
 * ||Y R - Zhat||_F, i.e. the orthogonal polar factor U V^T of Y^T Zhat
 * (Y, Zhat: n x d_s FP32), computed by a Newton-Schulz polar iteration in
 * FP32 until ||R^T R - I||_F < 1e-6.  Synchronises the stream.  Returns
 * ADANNS_ERR_ARG if Y^T Zhat is zero. */
int adanns_procrustes(const float *Y, const float *Zhat, int64_t n, int d_s, float *R,
                      void *cuda_stream);

/*
 * Train OPQ on the index's vectors and encode all of them (AdANNS-OPQ).
 *   db          the same N x d FP32 rows the index was built from (device).
 *   Training rows: first train_n entries of a splitmix64(seed + 2) shuffle of
 *   [0, N); Y = P_ds of those rows; R starts at I.  Each of opq_iters outer
 *   iterations: Z = Y R; pq_iters Lloyd steps per subspace (Forgy init from
 *   the rows at a splitmix64(seed + 3) shuffle of [0, train_n), codeword c
 *   taking entry c mod min(256, train_n), on the first iteration; warm start
 *   after); encode; R = Procrustes(Y, decode(codes)).  Then final_iters Lloyd
 *   steps on Y R, and every database vector is encoded.
 *   trace       optional HOST array of max(3 * opq_iters, 1) doubles: the mean
 *               squared distortion after each half-step (after the Lloyd
 *               steps, after the rotation update, after re-assigning under the
 *               new rotation; non-increasing up to FP32 rounding).
 * Synchronises the stream.  Replaces any OPQ data the index held.
 */
int adanns_build_opq(adanns_index *idx, const float *db, int d_s, int M, int opq_iters,
                     int pq_iters, int final_iters, int64_t train_n, uint64_t seed, double *trace,
                     void *cuda_stream);

/*
 * Residual-encoded AdANNS-IVFOPQ (the IVFOPQ row of Table "formula" with the
 * codes taken of residuals, the usual IVF-PQ variant; the paper does not
 * define it further).  The coarse centroids exist only at d_c, so the residual
 * of a database row x in list l is taken against that list's centre at d_s,
 * lcent[l] = the mean of P_ds over the list's members (FP64 sums, FP32
 * values; zero for an empty list): the codes quantise (P_ds(x) - lcent[l]) R.
 * adanns_build_opq_residual trains exactly as adanns_build_opq but on the
 * residuals of the training rows, and encodes every row's residual.  A search
 * (adanns_search_ivfopq, nprobe <= 256) then scores a member of a probed list
 * l by sum_m ||((P_ds(q) - lcent[l]) R)_m - C_m[code_m]||^2, evaluated as
 * sum_m (LUT_q[m][code_m] + S_l[m][code_m]) + |w_l|^2 - 2 <w_l, P_ds(q) R>
 * with w_l = lcent[l] R and S_l[m][c] = 2 <w_l,m, C_m[c]> (FP32 tables
 * nlist x M x 256 kept by the index; negative rounding residue is clamped to
 * 0).  adanns_index_set_opq_residual attaches given data (list_centres
 * [nlist][d_s] device FP32 plus what adanns_index_set_opq takes);
 * adanns_index_get_list_centres copies them out (ADANNS_ERR_STATE without
 * residual codes).  All three synchronise except the copy.
 */
int adanns_build_opq_residual(adanns_index *idx, const float *db, int d_s, int M, int opq_iters,
                              int pq_iters, int final_iters, int64_t train_n, uint64_t seed,
                              double *trace, void *cuda_stream);
int adanns_index_set_opq_residual(adanns_index *idx, int d_s, int M, const float *R,
                                  const float *codebooks, const uint8_t *codes_by_id,
                                  const float *list_centres, void *cuda_stream);
int adanns_index_get_list_centres(const adanns_index *idx, float *list_centres,
                                  void *cuda_stream);

/* Attach given OPQ data (device): R, codebooks and codes indexed by database
 * id (N x M); the codes are re-laid out in list order.  Synchronises. */
int adanns_index_set_opq(adanns_index *idx, int d_s, int M, const float *R,
                         const float *codebooks, const uint8_t *codes_by_id, void *cuda_stream);

/* Copy the index's OPQ data out (device buffers; any may be NULL); codes in
 * list order (row p belongs to the id at list position p).  ADANNS_ERR_STATE
 * if the index has no OPQ data. */
int adanns_index_get_opq(const adanns_index *idx, float *R, float *codebooks,
                         uint8_t *codes_list_order, void *cuda_stream);

/*
 * AdANNS-IVFOPQ search: the nprobe nearest centroids at d_c (as in
 * adanns_search_ivf); z = P_ds(q) R, LUT[m][c] = ||z_m - C_m[c]||^2; every
 * member of the probed lists scores sum_m LUT[m][code[m]]; the k best by
 * (score, id) are returned.  With rerank_k > 0 (k <= rerank_k <= 2048) the
 * rerank_k best by score are re-scored with the exact FP32 dist_ds of the
 * stored vectors and the k best of those are returned (Sec. 4.3
 * shortlist-rerank).  Outputs as adanns_search_ivf.  ADANNS_ERR_STATE if the
 * index has no OPQ data.  With nprobe <= 256 the scores are written to stream
 * scratch (4 bytes per member of the probed lists; the batch is sliced so
 * that this stays within the scratch budget) and the best are selected
 * afterwards; ADANNS_ADC_SELECT=0, or nprobe > 256, keeps a running top-k per
 * (query, list) instead.  Both give the same result.
 */
int adanns_search_ivfopq(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                         int nprobe, int k, int rerank_k, int64_t *out_ids, float *out_dist,
                         int32_t *out_probes, void *cuda_stream);

/* AdANNS-IVFOPQ search of a batch whose queries carry their own nprobe and k
 * (Sec. 5 compute-aware elastic search over the IVF-OPQ composite), in one
 * pass of the distance-then-select ADC stage.
 *   nprobe, k  HOST int32 arrays of B entries, read before the call returns:
 *            1 <= nprobe[i] <= min(nlist, 256), 1 <= k[i] <= k_max <= 1024.
 *   rerank_k 0, or k_max <= rerank_k <= 2048 (the shortlist of every query).
 *   out_ids  int64 [B x k_max], out_dist FP32 [B x k_max] (device): row i
 *            holds query i's k[i] results, then (-1, +inf) up to k_max.
 * Row i equals the first k[i] entries of adanns_search_ivfopq on query i alone
 * with (d_c, nprobe[i], k_max, rerank_k).  ADANNS_ERR_ARG for a bad entry (its
 * index in the message); nothing is launched then. */
int adanns_search_ivfopq_budgets(const adanns_index *idx, const float *queries, int64_t B,
                                 int d_c, const int32_t *nprobe, const int32_t *k, int k_max,
                                 int rerank_k, int64_t *out_ids, float *out_dist,
                                 void *cuda_stream);

/* ------------------------------------------------------------------------
 * Autotuning of the exact FP32 list scan.  adanns_autotune_search runs the
 * FP32 search of the given batch with each scan variant: the tiled scan with
 * 64 queries per (list, query-tile) item and a 4 x 8 register tile per thread
 * (k <= 128), the tiled scan with 16 queries and 1 x 8, and the streaming scan
 * (nprobe <= 256, ADANNS_OPT_FP32_STREAM on).  It times each with CUDA events
 * (1 warm-up, 3 timed runs; synchronises) and records the fastest for the
 * bucket (device, k rounded up to a power of two, d_s,
 * floor(log2(1 + B * nprobe / nlist))).  Later FP32 searches in the same
 * bucket use it.  All variants give the same results.  *chosen gets the winner
 * (4 or 1: the tiled scan's queries per thread; 16: the streaming scan),
 * *best_ms its time per call; both may be NULL.  out_ids / out_dist receive
 * the batch's results.  adanns_tune_save / adanns_tune_load write / merge the
 * table as text lines "<bucket key> <winner>".
 * ---------------------------------------------------------------------- */
int adanns_autotune_search(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                           int d_s, int nprobe, int k, int64_t *out_ids, float *out_dist,
                           void *cuda_stream, int *chosen, float *best_ms);
/*
 * Autotuning of the BF16 / FP8 tensor-core list scan's tile shape (the scan of
 * Algorithm 1 on the low-precision tier).  adanns_autotune_search_lowp runs
 * adanns_search_ivf of the given batch (storage ADANNS_STORE_BF16 or
 * ADANNS_STORE_FP8E4M3, rerank_k as there) once with tiles of 128 queries x
 * 256 members and once with tiles of 128 members x 32 queries, times each
 * with CUDA events (1 warm-up, 3 timed runs; synchronises) and records the
 * faster for the bucket (device, tier, d_s, floor(log2(1 + B * nprobe /
 * nlist))).  Later searches of that tier in the same bucket take the recorded
 * shape in place of the ADANNS_OPT_NARROW_SCAN = 1 rule.  The two shapes'
 * approximate keys agree up to the tensor cores' rounding of their dot
 * products; the exact rerank makes the returned distances exact either way.
 * *chosen gets 128 or 32 (queries per tile), *best_ms the time per call; both
 * may be NULL.  out_ids / out_dist receive the batch's results (last shape
 * run).  ADANNS_ERR_ARG for another storage or when ADANNS_OPT_NARROW_SCAN is
 * not 1 (a forced shape leaves nothing to tune).  The table is shared with
 * adanns_autotune_search (adanns_tune_save / adanns_tune_load).
 */
int adanns_autotune_search_lowp(const adanns_index *idx, const float *queries, int64_t B,
                                int d_c, int d_s, int nprobe, int k, int storage, int rerank_k,
                                int64_t *out_ids, float *out_dist, void *cuda_stream,
                                int *chosen, float *best_ms);
int adanns_tune_save(const char *path);
int adanns_tune_load(const char *path);
/* Forget every recorded choice (FP32 scan and tile shapes): later searches
 * take the built-in rules again. */
int adanns_tune_clear(void);

/* ------------------------------------------------------------------------
 * Search plans (batched search replayed from a captured CUDA graph).
 * adanns_plan_create runs adanns_search_ivf once with the given arguments on
 * cuda_stream (validating them, setting kernel attributes, growing the
 * scratch pool; synchronises), then captures the same call on a private
 * stream into a CUDA graph.  The plan is bound to the given device buffers:
 * each adanns_plan_launch re-runs the whole search (cluster mapping, probe
 * inversion, list scan, selection, rerank, merge) on the current contents of
 * `queries`, writing out_ids / out_dist, with one graph launch on
 * cuda_stream.  A plan may not run concurrently with itself.  Free it with
 * adanns_plan_free (waits for the device).
 * ---------------------------------------------------------------------- */
typedef struct adanns_plan adanns_plan;
int adanns_plan_create(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                       int nprobe, int k, int storage, int rerank_k, int64_t *out_ids,
                       float *out_dist, void *cuda_stream, adanns_plan **out);
int adanns_plan_launch(adanns_plan *plan, void *cuda_stream);
void adanns_plan_free(adanns_plan *plan);

/*
 * Size of the fixed device scratch array used by adanns_search_ivf_noalloc
 * (64 MiB, held on every GPU that loads this library until the process exits).
 */
#define ADANNS_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * AdANNS-IVF search that allocates no memory (not a step of the paper, which
 * has no counterpart; a deployment variant of adanns_search_ivf).
 *
 * For callers that cannot allocate device memory during a search: processes
 * whose framework has reserved the whole device memory budget for its own
 * pool, latency-critical loops where an allocator call that may synchronise
 * or grow a pool is not acceptable, or hosts whose policy forbids the library
 * from using the allocator.  It runs the FP32 search of adanns_search_ivf
 * (storage = ADANNS_STORE_F32, rerank_k = 0) with the same arguments, layouts
 * and error codes, but takes all scratch from one fixed file-scope device
 * array of ADANNS_NOALLOC_SCRATCH_BYTES.  It calls no cudaMalloc, cudaFree or
 * allocating routine.  It always takes the FP32 cluster mapping and the tiled
 * list scan with the default work shape (never the tensor-core cluster
 * mapping, the streaming scan, an autotuned shape or member-range splits), so
 * its results agree with adanns_search_ivf's within the FP32 tolerance of the
 * oracle comparison: distances within 1e-5 relative, ids equal except inside
 * groups of distances that tie within that tolerance.
 *
 * Scratch needed, each piece rounded up to 256 bytes:
 *   B*pad16(d_c)*4 + B*pad16(d_s)*4 + B*nprobe*8 + B*nprobe*k*8
 *   + 4*nlist*4 + 2*B*nprobe*4 + 3*T*4 + 4 + 8,  T = ceil(B*nprobe/QT) + nlist,
 * where QT (queries per work item) is 64 for k <= 128 and 16 above.  A request
 * that needs more returns ADANNS_ERR_ARG with the sizes in the message and
 * launches nothing.
 *
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Every call shares the one array and
 * leaves its contents behind (work counters are cleared by each call), so
 * calls that overlap on the GPU -- on different streams, or from several host
 * threads -- race and corrupt each other's results: serialise them.
 */
int adanns_search_ivf_noalloc(const adanns_index *idx, const float *queries, int64_t B, int d_c,
                              int d_s, int nprobe, int k, int64_t *out_ids, float *out_dist,
                              void *cuda_stream);

/* ------------------------------------------------------------------------
 * Low-d graph shortlist + high-d rerank (AdANNS-DiskANN, Sec. 4.3 "AdANNS for
 * Composite Indices": the search graph is formed with a low-d MR, its
 * shortlist is re-ranked with a high-d MR).
 *
 * adanns_graph_build forms a DiskANN-style pruned proximity graph on the d_g
 * prefix (P_dg under ADANNS_METRIC_L2_PREFIXNORM) of the N x d FP32 rows db
 * (device; copied, so the caller may free it): every row's K nearest other
 * rows (exact, ties to the lower id) are robust-pruned with factor alpha to at
 * most R out-neighbours (take the nearest remaining candidate c, drop every
 * remaining v with alpha * d(c, v) <= d(row, v)); every edge offers its
 * source to its target, and a row whose own and offered neighbours exceed R is
 * pruned again over their union by (distance, id).  The entry point is the
 * row nearest to the mean of the P_dg rows.  Limits: d_g in G and <= 64,
 * 1 <= R <= 64, 1 <= K <= 256, K < N, alpha >= 1; a row offered more than
 * 4,096 edges returns ADANNS_ERR_ARG.  Synchronises the stream.
 * adanns_graph_create takes a given graph instead (device int32 [N][R], -1
 * padding; an id outside [-1, N) returns ADANNS_ERR_ARG) and entry point.  adanns_graph_info / adanns_graph_get report it.
 *
 * adanns_graph_search: per query, a best-first search at d_g with a
 * candidate list of L entries (1 <= L <= 512) -- expand the nearest entry not
 * yet expanded, score its neighbours that are not in the list, keep the L
 * nearest by (distance, id) -- until every entry is expanded; the rerank_k
 * (k <= rerank_k <= min(L, 1024)) nearest entries are re-scored with the exact
 * FP32 dist_ds (d_s in G, <= d) and the k best by (distance, id) are returned
 * in out_ids / out_dist (device, [B][k], -1 / +inf padding); out_shortlist
 * (optional, device int64 [B][rerank_k]) receives the graph stage's list.
 * All distances are FP32 in difference form.  Asynchronous on the stream.
 */
typedef struct adanns_graph adanns_graph;
int adanns_graph_build(const float *db, int64_t N, int d, int d_g, int K, int R, float alpha,
                       int metric, void *cuda_stream, adanns_graph **out);
int adanns_graph_create(const float *db, int64_t N, int d, int d_g, const int32_t *graph, int R,
                        int64_t entry, int metric, void *cuda_stream, adanns_graph **out);
int adanns_graph_info(const adanns_graph *g, int64_t *N, int *d, int *d_g, int *R,
                      int64_t *entry);
int adanns_graph_get(const adanns_graph *g, int32_t *graph, void *cuda_stream);
int adanns_graph_search(const adanns_graph *g, const float *queries, int64_t B, int L, int d_s,
                        int k, int rerank_k, int64_t *out_ids, float *out_dist,
                        int64_t *out_shortlist, void *cuda_stream);
void adanns_graph_free(adanns_graph *g);

/* ------------------------------------------------------------------------
 * Continuous-batching server (the serving loop of the compute-aware elastic
 * search of Sec. 5 "Compute-aware Elastic Search During Inference": every
 * request carries its own compute budget over resident indices).
 *
 * adanns_server_create binds a server to the current device and to nindex
 * resident indices (not copied: they must outlive the server) and starts one
 * worker thread.  Requests are HOST query rows (n x d FP32 of the chosen
 * index; copied at submit, so the caller may reuse the buffer at once) with a
 * budget.  The worker keeps requests in arrival order; whenever one of its
 * nstreams CUDA streams is free it packs the oldest pending request with later
 * ones of the same index and budget into one batch of at most max_batch rows,
 * admits the batch if its scratch estimate (adanns_search_scratch_bytes plus
 * the batch's rows and results) fits mem_budget bytes next to the batches in
 * flight (a batch is always admitted when nothing is in flight), and runs it
 * on that stream: pinned staging, host-to-device copy, the search,
 * device-to-host copy of the results.  Batches on different streams overlap
 * on the device.  A request's rows get the same ids and distances as the same
 * rows searched alone with adanns_search_ivf / adanns_search_ivfopq.
 *
 * adanns_server_submit checks the budget against the index (the search's own
 * argument rules; errors are returned there) and returns a ticket.
 * adanns_server_poll waits up to wait_ms (0: no wait, -1: until done) for the
 * ticket; it returns ADANNS_PENDING (1) if the request is not finished, else
 * retires the ticket and returns ADANNS_OK with the results copied to the HOST
 * arrays ids (int64 [n][k]) and dist (FP32 [n][k]) and the latency from submit
 * to results on the host, or the error the request's batch met (message in
 * adanns_last_error on the polling thread).  adanns_server_stats reports
 * latency percentiles (p50, p99 over finished requests), requests launched,
 * batches, rows served, rows per second between the first submit and the last
 * completion, and the largest memory estimate in flight; any pointer may be
 * NULL.  adanns_server_destroy stops accepting requests, finishes the pending
 * and in-flight ones, stops the worker and frees the server (results not
 * polled are dropped); no other call on the server may run concurrently with
 * it.  Submit, poll and stats may be called from any threads.
 * ---------------------------------------------------------------------- */
#define ADANNS_PENDING 1
#define ADANNS_METHOD_IVF 0    /* adanns_search_ivf with the budget's storage tier */
#define ADANNS_METHOD_IVFOPQ 1 /* adanns_search_ivfopq (d_s and storage unused) */

typedef struct adanns_budget {
  int method;   /* ADANNS_METHOD_* */
  int d_c, d_s, nprobe, k;
  int storage;  /* ADANNS_STORE_F32 / _BF16 / _FP8E4M3 for ADANNS_METHOD_IVF */
  int rerank_k; /* as in the search calls */
} adanns_budget;

typedef struct adanns_server adanns_server;
int adanns_server_create(const adanns_index *const *indices, int nindex, int nstreams,
                         int64_t max_batch, int64_t mem_budget, adanns_server **out);
int adanns_server_submit(adanns_server *srv, int index_slot, const float *queries, int64_t n,
                         const adanns_budget *budget, int64_t *ticket);
int adanns_server_poll(adanns_server *srv, int64_t ticket, int wait_ms, int64_t *ids, float *dist,
                       double *latency_ms);
int adanns_server_stats(adanns_server *srv, double *p50_ms, double *p99_ms, int64_t *requests,
                        int64_t *batches, int64_t *queries, double *qps, int64_t *max_inflight);
int adanns_server_destroy(adanns_server *srv);

/* ------------------------------------------------------------------------
 * Lists partitioned over several GPUs (the IVF probe/scan is independent per
 * inverted list, Alg. 1 and Sec. 4.2, so the lists can live on different
 * devices; the per-device top-k of one query are then merged by distance).
 * Each device holds an index over the rows of the lists it owns, with the
 * full centroid table, so every device probes the same n_p lists and scans
 * the owned ones.  These two calls are the device steps of the merge; the
 * exchange of the per-device results between devices is the caller's.
 * ---------------------------------------------------------------------- */

#define ADANNS_MAX_SHARDS 128

/*
 * In place: ids[i] = map[ids[i]] for 0 <= ids[i] < n_map; negative ids
 * (padding) are kept; ids >= n_map (impossible for results of a search of an
 * index over n_map rows) become -1.
 *   map    device, n_map int64: global id of each local row, ascending if the
 *          merged result is to break distance ties by global id exactly as a
 *          single-device search does
 *   ids    device, count int64, read and written on the stream
 * Errors: ADANNS_ERR_ARG for negative sizes or NULL pointers with count > 0.
 * Asynchronous on cuda_stream.
 */
int adanns_map_ids(const int64_t *map, int64_t n_map, int64_t *ids, int64_t count,
                   void *cuda_stream);

/*
 * Merge of G per-shard top-k results into one top-k per query, by (distance,
 * id) ascending; fewer than k valid entries overall pad with (-1, +inf).
 *   ids, dist  device, [G][B][k] (shard-major) int64 / float32; each row
 *              sorted ascending by (distance, id) with padding (id < 0) at its
 *              end, as adanns_search_ivf returns it; ids below 2^32 - 1
 *   out_ids, out_dist  device, [B][k], written on the stream
 * An id that appears in several shards appears that many times (shards are
 * expected to be disjoint).
 * Errors: ADANNS_ERR_ARG unless 1 <= G <= ADANNS_MAX_SHARDS, 1 <= k <= 1024,
 * 0 <= B <= 2^31 - 1, and (for B > 0) no pointer is NULL.
 * Asynchronous on cuda_stream.
 */
int adanns_merge_shards(const int64_t *ids, const float *dist, int G, int64_t B, int k,
                        int64_t *out_ids, float *out_dist, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ADANNS_H */
