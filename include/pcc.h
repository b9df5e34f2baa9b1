/*
 * pcc.h -- C ABI of the GB300 all-pairs Pearson correlation library.
 *
 * The library computes, for an n x l matrix X of n variables (genes) with
 * l samples each, the Pearson correlation r(i,j) of every pair of rows,
 * Eq. (1) of LightPCC (Liu, Pan and Aluru, arXiv 1605.01584, Section I):
 *
 *   r(u,v) = sum_k (u_k - ubar)(v_k - vbar)
 *            / sqrt( sum_k (u_k - ubar)^2 * sum_k (v_k - vbar)^2 )
 *
 * through the paper's reformulation (Section III-A, Eq. (5)-(6)): each row
 * is centred and scaled to unit norm once, z_i = (x_i - xbar_i)/||x_i -
 * xbar_i||, after which r(i,j) = z_i . z_j, the upper triangle of Z Z^T.
 *
 * Conventions shared by every entry point:
 *   - Data pointers (X, R, edges, counts, permutations) are DEVICE pointers
 *     owned by the caller; the library never frees them.  A pcc_zmat is
 *     allocated by the library (pcc_standardize) and released with
 *     pcc_zmat_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call only enqueues work on that stream and returns;
 *     results are ready once the stream is synchronised.
 *   - Calls return a pcc_status and never abort, trap or throw.  Errors the
 *     GPU detects while running (a pipeline wait that exceeded its limit, an
 *     edge list that overflowed) are recorded in a status word inside the
 *     pcc_zmat and returned by pcc_sync_status.
 *   - Row-major layouts with explicit leading dimensions; sizes are int64.
 *   - Pairs are i < j (the major diagonal is excluded, Section III-B allows
 *     this adaptation).  The packed output holds pair (i,j) at
 *       J(i,j) = i(2n - i - 1)/2 + (j - i - 1)
 *     (Eq. (9)-(10) of Section III-B with the diagonal removed), so the
 *     pairs of row i are contiguous and rows follow each other.
 *   - A row whose centred sum of squares is zero or not finite is flagged;
 *     every r involving it is NaN (Eq. (1) gives 0/0), it never becomes an
 *     edge and its permutation count is 0.
 */
#ifndef PCC_H
#define PCC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PCC_OK = 0,
    PCC_ERR_INVALID_ARG = 1, /* bad size, pointer, range or combination */
    PCC_ERR_CUDA = 2,        /* a CUDA runtime/driver call failed */
    PCC_ERR_OOM = 3,         /* device allocation failed */
    PCC_ERR_CAPACITY = 4,    /* edge list longer than its capacity */
    PCC_ERR_TIMEOUT = 5,     /* a device pipeline wait exceeded its limit */
    PCC_ERR_UNSUPPORTED = 6, /* no kernel for this device / combination */
    PCC_ERR_ABORTED = 7      /* a caller's callback asked to stop */
} pcc_status;

/* element type of an input or output array */
typedef enum { PCC_F32 = 0, PCC_F64 = 1 } pcc_dtype;

/* Forms of the permutation test (pcc_set_perm_form); all give the same
 * counts. */
typedef enum {
    PCC_PERM_SMEM = 0,       /* CTA pairs permute resident rows in shared
                                memory */
    PCC_PERM_WORKSPACE = 1,  /* a gather launch writes permuted rows to a
                                work buffer first */
    PCC_PERM_TRANSPOSED = 2  /* CTA pairs copy permuted operands from a
                                transposed copy of Z (the default) */
} pcc_perm_form;

/* how Z is stored and which pair kernel contracts it */
typedef enum {
    PCC_PREC_FP64 = 0,    /* Z in FP64; FP64 CUDA-core pair kernel */
    PCC_PREC_FP32 = 1,    /* Z in FP32; FP32 CUDA-core pair kernel */
    PCC_PREC_BF16X3 = 2,  /* Z = hi + lo, both BF16; tensor cores run
                             hi.hi + hi.lo + lo.hi, FP32 accumulation */
    PCC_PREC_FP16X3S = 3, /* as BF16X3 with FP16 halves of z * 2^s,
                             s = floor(log2(l)/2); about 30x more accurate */
    PCC_PREC_BF16X4 = 4,  /* as BF16X3 plus the lo.lo product (4 MMAs per
                             K step instead of 3) */
    PCC_PREC_BF16X1 = 5,  /* Z = bf16(z), one product (reported only:
                             about 1e-3 error) */
    PCC_PREC_AUTO = 6     /* the split form with the smaller worst-case
                             error: FP16X3S at every l (on rows whose mass
                             sits in one sample BF16X3's BF16 halves alone
                             reach 1.0-1.3e-5; FP16X3S stays within 1e-5,
                             with long rows accumulated in chunks of at
                             most 640 samples) */
} pcc_prec;

typedef struct pcc_zmat pcc_zmat; /* opaque, library-owned */

/* one |r| >= tau edge, i < j, r signed (12 bytes) */
typedef struct {
    uint32_t i, j;
    float r;
} pcc_edge;

/* ------------------------------------------------------------------ */
/* Step 1: variable transformation (Eq. (5), Algorithm 3).             */
/* ------------------------------------------------------------------ */

/* Centre and scale every row of X to unit norm: per row, the mean and the
 * centred sum of squares S are accumulated in FP64 (two passes, as
 * Algorithm 3), then z = (x - mean)/sqrt(S) is stored in the form `prec`
 * asks for (PCC_PREC_AUTO is resolved here).
 *   X    device, n x l, row-major, leading dimension ldx >= l, element type
 *        xt (PCC_F32 or PCC_F64).
 *   *Z   if *Z is non-NULL and was made for the same device, n, l and
 *        precision it is overwritten in place (no allocation); otherwise a
 *        new pcc_zmat is allocated and returned in *Z (an old one is left
 *        to the caller to destroy).
 * Errors: PCC_ERR_INVALID_ARG for n < 2, l < 2, ldx < l, n >= 2^31, NULL X
 * or Z; PCC_ERR_OOM; PCC_ERR_UNSUPPORTED for tensor-core forms on a device
 * that is not sm_103. */
pcc_status pcc_standardize(const void *X, pcc_dtype xt, int64_t n, int64_t l,
                           int64_t ldx, pcc_prec prec, pcc_zmat **Z,
                           void *stream);

/* pcc_standardize from a HOST matrix (Eq. (5), Algorithm 3, as above):
 * the call copies X_host (host memory, n x l, leading dimension ldx >= l,
 * element type xt) into a device copy owned by *Z, then standardizes it on
 * `stream`.  With pinned (page-locked) X_host the copy is asynchronous and
 * X_host must stay unchanged until the stream reaches it; with pageable
 * memory the copy completes before the call returns.  The device copy is
 * allocated by the first call that needs it (or a larger one) and reused
 * after, so later calls of the same size allocate nothing.  This is the
 * entry of a program whose data start in host memory (the paper's offload
 * model, Section III-C: input sent once, results streamed back).
 * Errors: as pcc_standardize, PCC_ERR_INVALID_ARG for a NULL X_host. */
pcc_status pcc_standardize_host(const void *X_host, pcc_dtype xt, int64_t n,
                                int64_t l, int64_t ldx, pcc_prec prec,
                                pcc_zmat **Z, void *stream);

/* pcc_standardize for B FP32 matrices at once (Eq. 5 / Algorithm 3 applied
 * to each; the batching is this library's, for the many-datasets workload):
 * one launch per stored form covers up to 96 matrices, each with its own
 * n, l and pitch, so small matrices do not each pay a launch.  The results
 * are the same bits as B pcc_standardize calls.
 *   Xs[b]   device, ns[b] x ls[b] FP32, row-major, leading dimension
 *           ldxs[b] >= ls[b]; the arrays Xs, ns, ls, ldxs, Zs are host
 *           arrays of B entries.
 *   Zs[b]   as pcc_standardize's *Z: reused when it matches (device, n, l,
 *           precision), otherwise replaced by a new pcc_zmat (an old one is
 *           left to the caller).  prec applies to every matrix (AUTO is
 *           resolved per matrix from its l).
 * Errors: PCC_ERR_INVALID_ARG for B < 1, a NULL array or X, or any matrix
 * pcc_standardize would reject (checked before anything is allocated or
 * launched); PCC_ERR_OOM (the Zs created so far are returned);
 * PCC_ERR_UNSUPPORTED as pcc_standardize. */
pcc_status pcc_standardize_batched(const float *const *Xs, const int64_t *ns,
                                   const int64_t *ls, const int64_t *ldxs,
                                   int32_t B, pcc_prec prec, pcc_zmat **Zs,
                                   void *stream);

/* Free a pcc_zmat (waits for nothing: the caller must have synchronised
 * the streams that use it).  NULL is accepted. */
pcc_status pcc_zmat_destroy(pcc_zmat *Z);

/* Shape and form of Z: n, l, padded row length lpad (elements), resolved
 * precision, and the power-of-two exponent s of PCC_PREC_FP16X3S (0
 * otherwise).  Any output pointer may be NULL. */
pcc_status pcc_zmat_info(const pcc_zmat *Z, int64_t *n, int64_t *l,
                         int64_t *lpad, int32_t *prec, int32_t *scale_exp);

/* Device pointers to Z's storage (read-only views, owned by Z): hi and lo
 * (2-byte halves, n x lpad) for the split forms, z (FP32 or FP64, n x lpad)
 * otherwise, flags (n bytes, 1 = zero-variance or non-finite row).
 * Pointers that do not apply are set to NULL. */
pcc_status pcc_zmat_buffers(const pcc_zmat *Z, const void **hi,
                            const void **lo, const void **z,
                            const uint8_t **flags);

/* ------------------------------------------------------------------ */
/* Step 2: all pairs (Eq. (6); tiles scheduled by Eq. (16)-(19)).       */
/* ------------------------------------------------------------------ */

/* Number of work tiles of Z's pair schedule (the unit of tile ranges). */
int64_t pcc_num_tiles(const pcc_zmat *Z);

/* Packed strict upper triangle: R[J(i,j)] = r(i,j) for all i < j covered
 * by tiles [tile_begin, tile_end) of Z's schedule (tile_end = -1 means
 * pcc_num_tiles(Z)); other entries of R are not touched, so disjoint tile
 * ranges can be computed by different calls, devices or ranks (Section
 * III-D distributes equal ranges of tile ids).
 *   R   device, n(n-1)/2 elements of type rt.  rt = PCC_F64 only for
 *       PCC_PREC_FP64.  Tensor-core forms clamp r to [-1, 1].
 * Errors: PCC_ERR_INVALID_ARG for NULL, a bad range or dtype. */
pcc_status pcc_allpairs_upper(const pcc_zmat *Z, void *R, pcc_dtype rt,
                              int64_t tile_begin, int64_t tile_end,
                              void *stream);

/* Co-expression edges: every pair with |r(i,j)| >= tau (inclusive, either
 * sign; flagged rows never qualify) is appended to `edges` in an
 * unspecified order, through one atomic per warp on *d_count.
 *   edges     device, room for `capacity` records (may be NULL if
 *             capacity == 0).
 *   d_count   device uint64, ADDED to (the caller zeroes it first); after
 *             the call it holds the true number of qualifying pairs even
 *             when that exceeds capacity, in which case only `capacity` of
 *             them are stored and pcc_sync_status reports
 *             PCC_ERR_CAPACITY.
 *   R         optional device FP32 packed output written in the same pass
 *             (NULL = edges only).  Needs a tensor-core or FP32 Z. */
pcc_status pcc_threshold_edges(const pcc_zmat *Z, float tau, pcc_edge *edges,
                               uint64_t capacity, uint64_t *d_count,
                               float *R, void *stream);

/* ------------------------------------------------------------------ */
/* Non-symmetric all pairs between two matrices (Section III-B,        */
/* Eq. (7)-(8)): r(x_i, y_j) for every row x_i of X and y_j of Y.       */
/* ------------------------------------------------------------------ */

/* Number of work tiles of the cross schedule of ZX against ZY (the unit of
 * tile ranges); -1 if either is NULL. */
int64_t pcc_cross_num_tiles(const pcc_zmat *ZX, const pcc_zmat *ZY);

/* Dense cross-correlation: R[i * ldr + j] = r(x_i, y_j) for 0 <= i < nx,
 * 0 <= j < ny, over tiles [tile_begin, tile_end) of the cross schedule
 * (tile_end = -1: all of them); other entries are not touched.
 *   ZX, ZY  standardized by pcc_standardize on one device with the same l
 *           and the same (resolved) form; ZX may equal ZY (the full square
 *           matrix, diagonal included).
 *   R       device, nx rows of ldr >= ny elements of type rt (PCC_F64 only
 *           for PCC_PREC_FP64).  Flagged rows give NaN; tensor-core forms
 *           clamp to [-1, 1].
 * Errors: PCC_ERR_INVALID_ARG for NULL, mismatched Z's, ldr < ny, a bad
 * range or dtype. */
pcc_status pcc_cross_allpairs(const pcc_zmat *ZX, const pcc_zmat *ZY,
                              void *R, pcc_dtype rt, int64_t ldr,
                              int64_t tile_begin, int64_t tile_end,
                              void *stream);

/* Cross edges: every (i, j) with |r(x_i, y_j)| >= tau is appended as
 * {i, j, r} (i indexes X, j indexes Y), with the same count and capacity
 * rules as pcc_threshold_edges; R (FP32, pitch ldr, or NULL) is written in
 * the same pass.  Not for PCC_PREC_FP64 with R. */
pcc_status pcc_cross_edges(const pcc_zmat *ZX, const pcc_zmat *ZY, float tau,
                           pcc_edge *edges, uint64_t capacity,
                           uint64_t *d_count, float *R, int64_t ldr,
                           void *stream);

/* ------------------------------------------------------------------ */
/* Outputs larger than the device: passes with asynchronous copies     */
/* (Section III-C's multi-pass execution, Algorithm 2).                 */
/* ------------------------------------------------------------------ */

/* Called on the calling thread once rows [row_begin, row_end) of the output
 * are complete in host memory at `rows` (their packed slice, or for the
 * cross form their dense rows), while the device computes the next pass.
 * A non-zero return stops the computation (PCC_ERR_ABORTED). */
typedef int32_t (*pcc_rows_sink)(void *user, int64_t row_begin,
                                 int64_t row_end, const void *rows);

/* The packed strict upper triangle of Z (as pcc_allpairs_upper) delivered
 * to HOST memory in passes of whole row blocks, each computed into one of
 * two device windows and copied out while the next pass computes.
 *   R_host        host, n(n-1)/2 elements of type rt (pinned memory lets
 *                 the copies overlap the kernels); NULL = no host copy of
 *                 the whole triangle: each slice is staged in a
 *                 library-owned pinned buffer, valid during the sink call.
 *   device_bytes  bytes for the two windows (<= 0: a quarter of the free
 *                 device memory, at most 4 GiB).
 *   sink          may be NULL when R_host is given.
 * Errors: PCC_ERR_INVALID_ARG (no R_host and no sink, bad dtype);
 * PCC_ERR_OOM when one row block does not fit the budget;
 * PCC_ERR_ABORTED.  Returns after the last slice was delivered; kernel
 * status (timeouts) is read with pcc_sync_status. */
pcc_status pcc_allpairs_upper_host(const pcc_zmat *Z, void *R_host,
                                   pcc_dtype rt, int64_t device_bytes,
                                   pcc_rows_sink sink, void *user,
                                   void *stream);

/* pcc_threshold_edges with R delivered to host memory the same way: the
 * edge list (device, as pcc_threshold_edges) and the FP32 packed triangle
 * (R_host or the sink's staged slices) come from the same passes.  Not for
 * PCC_PREC_FP64. */
pcc_status pcc_threshold_edges_host(const pcc_zmat *Z, float tau,
                                    pcc_edge *edges, uint64_t capacity,
                                    uint64_t *d_count, float *R_host,
                                    int64_t device_bytes, pcc_rows_sink sink,
                                    void *user, void *stream);

/* The same for the dense cross matrix: R_host rows of pitch ldr >= ny (a
 * staged slice has pitch ny). */
pcc_status pcc_cross_allpairs_host(const pcc_zmat *ZX, const pcc_zmat *ZY,
                                   void *R_host, pcc_dtype rt, int64_t ldr,
                                   int64_t device_bytes, pcc_rows_sink sink,
                                   void *user, void *stream);

/* Bring an edge list to host memory: synchronises `stream`, stores the
 * device count (*d_count, as written by the edge calls) in *count_host and
 * copies the first min(count, capacity) records of `edges` (device) to
 * edges_host (host, capacity records).  Returns PCC_ERR_CAPACITY when the
 * count exceeds capacity (the records that fit are copied), else PCC_OK;
 * PCC_ERR_INVALID_ARG for NULL d_count or count_host, or NULL edges /
 * edges_host with capacity > 0.  The co-expression network of Section I,
 * delivered to the host. */
pcc_status pcc_edges_copy_host(const pcc_edge *edges, const uint64_t *d_count,
                               uint64_t capacity, pcc_edge *edges_host,
                               uint64_t *count_host, void *stream);

/* Permutation test (Section IV-A): for permutations k in [k0, k1) of the P
 * given ones, r_k(i,j) = z_i . (z_j o pi_k) with (z_j o pi_k)[s] =
 * z_j[pi_k[s]] (only the second row of a pair is permuted); d_counts[J(i,j)]
 * is INCREASED by #{k : |r_k(i,j)| >= |r(i,j)|}.  Counting a range and
 * adding lets a long test be split or resumed.
 *   d_perms   device int32, P x l, row k a permutation of 0..l-1.  Each
 *             index is checked on the device: one outside [0, l) is read as
 *             sample 0 and recorded as PCC_ERR_INVALID_ARG in Z's status
 *             (pcc_sync_status).  Whether a row is a permutation is not
 *             checked.
 *   d_counts  device uint32, n(n-1)/2, packed like R.
 * Three forms, with the same counts (pcc_set_perm_form):
 *   - the transposed form (the default; CTA pairs, rows of up to 256 padded
 *     samples): the first call after each standardize writes a transposed
 *     copy of Z (2 x lpad x n 16-bit values, kept in Z), so that the
 *     permuted column operand of a tile is a set of rows of that copy,
 *     which the kernel copies from L2 into shared memory as it goes.  A
 *     call recorded by a stream capture always rebuilds the copy (a replay
 *     may follow a later standardize).  The first call on a Z allocates
 *     the copy: make it before capturing;
 *   - the workspace form: the permuted rows of a batch of permutations are
 *     first written to a work buffer, allocated by the first such call on a
 *     Z and kept in Z (4.2 GB for 1,000 permutations of a 4,096 x 256
 *     matrix; smaller budgets run in batches; make the first call before
 *     capturing); about 1.1 to 1.2 times the transposed form's time;
 *   - the shared-memory form (CTA pairs, rows of up to 256 padded samples):
 *     each CTA keeps 64 of the column tile's rows z_j resident in shared
 *     memory and builds every permuted operand there; no device memory is
 *     allocated, at about 3 times the transposed form's time.
 * Errors: PCC_ERR_INVALID_ARG for a bad range, NULL pointers or a non
 * tensor-core Z. */
pcc_status pcc_perm_test(const pcc_zmat *Z, const int32_t *d_perms,
                         int32_t P, int32_t k0, int32_t k1,
                         uint32_t *d_counts, void *stream);

/* All pairs of B independent matrices of uneven n and l in one persistent
 * launch: Rs[b] (device, n_b(n_b-1)/2 floats) receives the packed FP32
 * triangle of Zs[b].  All Zs are tensor-core forms on one device; each may
 * use its own split form.  The work units of all matrices are spread over
 * the CTAs longest first by a cost model (pcc_set_tuning).  The first call
 * with a given set of (Zs, Rs) builds and caches a device work list (a small
 * allocation); later calls with the same set allocate nothing, so make the
 * first one before capturing a stream.  Device errors are reported in
 * Zs[0]'s status word.
 * Errors: PCC_ERR_INVALID_ARG for B < 1, NULL entries, a non tensor-core Z
 * or Zs on different devices; PCC_ERR_OOM. */
pcc_status pcc_allpairs_upper_batched(const pcc_zmat *const *Zs, int32_t B,
                                      float *const *Rs, void *stream);

/* pcc_allpairs_upper_batched with a choice per matrix (the tuner's, for
 * each matrix's shape; the paper has no counterpart):
 *   pair[b]       1: matrix b runs on CTA pairs as 2-SM MMAs, 0: on single
 *                 CTAs (NULL: the current pcc_set_pair_mma / cluster knob
 *                 for every matrix);
 *   band_rows[b]  super-tile rows per band of matrix b's order, 1..4096
 *                 (NULL: the current band_rows for every matrix).
 * One kernel issues either 2-SM or 1-SM MMAs, so the matrices of each form
 * run in one persistent launch of their own: one launch when all share a
 * form, two (pair form first, both on `stream`) otherwise.  Each matrix's
 * result has the bits of a pcc_allpairs_upper of it under the same form and
 * band rows.  The work list is built and cached as in
 * pcc_allpairs_upper_batched (per set of Zs, Rs and choices).
 * Errors: as pcc_allpairs_upper_batched, and PCC_ERR_INVALID_ARG for a pair
 * value other than 0 or 1 or a band_rows value out of range. */
pcc_status pcc_allpairs_upper_batched_tuned(const pcc_zmat *const *Zs,
                                            int32_t B, float *const *Rs,
                                            const int32_t *pair,
                                            const int32_t *band_rows,
                                            void *stream);

/* All pairs without any device allocation (the paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory,
 * e.g. code running inside another framework's memory pool, programs with
 * a device-memory budget fixed at start-up, or latency-critical paths that
 * cannot afford cudaMalloc's implicit synchronisation).
 * Standardizes X (device FP32, n x l, leading dimension ldx) and writes the
 * packed FP32 triangle R (device, n(n-1)/2 floats) as pcc_standardize +
 * pcc_allpairs_upper do, but keeps the standardized matrix in one
 * file-scope device array of 32 MiB that every device holds from the time
 * it loads the library until the process exits.
 *   prec      PCC_PREC_BF16X3, PCC_PREC_FP16X3S, PCC_PREC_BF16X4,
 *             PCC_PREC_BF16X1 or
 *             PCC_PREC_AUTO (tensor-core forms only).
 *   d_status  optional device int32 (caller-owned, may be NULL) set to 0 by
 *             the call and then to PCC_ERR_TIMEOUT if a device wait ran out.
 *             With NULL the status goes to a word inside the array that no
 *             call returns: a timeout is then not reported, and R may be
 *             left partly written, so pass d_status wherever failures must
 *             be seen.
 * Limit: 4 * n * lpad + n (rounded up to 256) + 256 <= 32 MiB, with lpad = l
 * rounded up to 64 (e.g. n = 16384 with l <= 448, or n = 8192 with l <=
 * 960); larger problems return PCC_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address (no
 * allocation); make that first call before any stream capture.  All calls
 * on a device share the array, so calls that may overlap on the GPU (on
 * unordered streams) race: order them on one stream. */
pcc_status pcc_allpairs_upper_noalloc(const float *X, int64_t n, int64_t l,
                                      int64_t ldx, pcc_prec prec, float *R,
                                      int32_t *d_status, void *stream);

/* Synchronise `stream`, then return and clear the device status word of Z
 * (PCC_OK, PCC_ERR_TIMEOUT or PCC_ERR_CAPACITY). */
pcc_status pcc_sync_status(pcc_zmat *Z, void *stream);

/* Knobs of the tensor-core kernels, as chosen by the tuner
 * (paper_1605_01584_gb300/autotune.py); they affect later launches only and
 * never the result.  0 (or <= 0 for the costs) keeps a value.
 *   stage_k    K per shared-memory ring stage: 32 (4 stages; 6 in the 2-SM
 *              pair form, whose stages are a third smaller) or 64 (2; 3 in
 *              the pair form; the default, PCC_TC_BK=32 in the environment
 *              selects 32 when the library loads).  The batched kernel
 *              follows it too.  The permutation test's workspace form
 *              follows it with CTA pairs (single CTAs keep 32); its
 *              shared-memory form always stages 32.
 *   cluster    2 = CTA pairs running one 2-SM MMA (while
 *              pcc_set_pair_mma is on), 1 = independent CTAs.
 *   band_rows  super-tile rows per band of the pair schedule (rows of a
 *              band stay in L2 while column panels stream once per band).
 *   cost_c0, cost_c1  cost model of pcc_allpairs_upper_batched's work
 *              split: cycles per work unit outside the K loop and per K
 *              block of 32 per product.
 * Errors: PCC_ERR_INVALID_ARG for a value out of range (nothing changes).
 * The paper has no counterpart (its tile size t is fixed at 4). */
pcc_status pcc_set_tuning(int32_t stage_k, int32_t cluster, int32_t band_rows,
                          double cost_c0, double cost_c1);

/* The CTA-pair form of the tensor-core kernels.  on = 1 (the default;
 * PCC_TC_PAIR=0 in the environment selects 0 when the library loads): two
 * CTAs run one 2-SM MMA (tcgen05.mma.cta_group::2, M = 256 rows over both),
 * each loading only half of the column operand, which the pair's tensor
 * cores exchange.  on = 0: independent CTAs, each loading its whole
 * operands.  No form copies an operand to several CTAs (no TMA multicast).
 *   pcc_allpairs_upper / _edges / cross (cluster = 2): the
 *   pair computes one 256 x 256 super-tile; on = 0: each CTA computes a
 *   128 x 256 half on its own.
 *   pcc_perm_test: the pair computes two 128 x 128 tiles of one tile
 *   column, each CTA loading one of the two permutations of a pass; on = 0:
 *   independent CTAs, one tile each.
 *   pcc_allpairs_upper_batched: CTA pairs take whole super-tiles; on = 0:
 *   independent CTAs take halves.
 * Affects later launches only; the results are the same bits.  Errors:
 * PCC_ERR_INVALID_ARG unless on is 0 or 1.  The paper has no counterpart
 * (a GB300 execution choice). */
pcc_status pcc_set_pair_mma(int32_t on);
int32_t pcc_get_pair_mma(void);

/* The form of pcc_perm_test (a pcc_perm_form; PCC_PERM_FORM=<0|1|2> in the
 * environment sets it when the library loads).  PCC_PERM_TRANSPOSED (the
 * default) and PCC_PERM_SMEM apply where rows fit (padded length <= 256),
 * pcc_set_pair_mma is on and n > 128; elsewhere the workspace form runs.
 * Affects later calls only; the counts are the same.
 * Errors: PCC_ERR_INVALID_ARG unless form is 0, 1 or 2.  The paper has no
 * counterpart (a GB300 execution choice). */
pcc_status pcc_set_perm_form(int32_t form);
int32_t pcc_get_perm_form(void);

/* Current knob values (any pointer may be NULL). */
pcc_status pcc_get_tuning(int32_t *stage_k, int32_t *cluster,
                          int32_t *band_rows, double *cost_c0,
                          double *cost_c1);

/* Measure the FP32 fused multiply-add rate of the current device's CUDA
 * cores (TFLOP/s, 2 flops per FMA), the roofline of the CUDA-core pair
 * kernels (the FP32 form is the comparison path of the split tensor-core
 * forms).  Runs a kernel of independent FMA chains on `stream` (8 blocks of
 * 256 threads per SM, best of three timed launches) and waits for it; it
 * allocates nothing.  Errors: PCC_ERR_INVALID_ARG for a NULL tflops,
 * PCC_ERR_CUDA.  The paper has no counterpart (a measurement helper). */
pcc_status pcc_measure_fp32_fma(double *tflops, void *stream);

/* Limit, in nanoseconds, of every pipeline wait inside the tensor-core
 * kernels (default 4e9).  A wait that runs out sets PCC_ERR_TIMEOUT in the
 * status word and the kernel returns early instead of hanging. */
pcc_status pcc_set_wait_limit_ns(uint64_t ns);

/* Test hook for the failure path (the paper has no counterpart).  It acts
 * on the tensor-core pair kernel and on the shared-memory form of
 * pcc_perm_test (whose producer loads the A rows).
 *   enable = 1  the TMA producer issues no loads, so every CTA's first
 *               operand wait runs out after the wait limit;
 *   enable = 2  in the CTA-pair form only the odd CTA of each pair issues
 *               none (the even CTA's copies land, its MMA waits for the
 *               odd CTA's share and runs out);
 *   enable = 3  only the even CTA issues none (the odd CTA's copies land on
 *               barriers the even CTA never armed);
 *   enable = 0  off.
 * The kernel records PCC_ERR_TIMEOUT, waits (bounded) until every copy that
 * was issued has landed, frees its TMEM and returns, and the CUDA context
 * stays usable.  Nothing faults or hangs.  Pair with a short
 * pcc_set_wait_limit_ns.  Never enable it outside tests.
 * Errors: PCC_ERR_INVALID_ARG unless 0 <= enable <= 3. */
pcc_status pcc_debug_drop_loads(int32_t enable);

/* ------------------------------------------------------------------ */
/* Numbering helpers (host functions, Section III-B/C).                */
/* ------------------------------------------------------------------ */

/* n(n-1)/2, 0 for n < 2 */
int64_t pcc_num_pairs(int64_t n);

/* J(i,j) above for 0 <= i < j < n, else -1 */
int64_t pcc_pair_index(int64_t n, int64_t i, int64_t j);

/* inverse of pcc_pair_index by the closed form of Eq. (14)-(15) (with n
 * replaced by n-1 for the strict triangle) in FP64 followed by an exact
 * integer correction; PCC_ERR_INVALID_ARG if J is out of range */
pcc_status pcc_pair_coords(int64_t n, int64_t J, int64_t *i, int64_t *j);

/* Eq. (17)-(19): tile id Jt in [0, m(m+1)/2) -> (yt, xt), yt <= xt, by the
 * same closed form plus correction the kernels use */
pcc_status pcc_tile_coords(int64_t m, int64_t Jt, int64_t *yt, int64_t *xt);

/* The tile schedule of the pair kernels, on the host (no device needed):
 * pcc_schedule_num_tiles(n, prec) = pcc_num_tiles of a Z of n rows stored
 * in form prec (AUTO resolved as pcc_standardize does), or -1 for n < 2 or
 * a bad prec; pcc_schedule_tile_rect gives tile `tile`'s rows [row0, row1)
 * and columns [col0, col1), clipped to n: the pairs i < j inside it are the
 * ones pcc_allpairs_upper(Z, R, tile, tile + 1) writes.  Tensor-core forms
 * follow the banded super-tile order with the current band_rows
 * (pcc_set_tuning: keep it unchanged between computing and reading a tile
 * range), the CUDA-core forms the triangular tile order of Eq. (17)-(19).
 * This is how the ranks of Section III-D's distribution know which packed
 * runs each of them wrote.  PCC_ERR_INVALID_ARG for an id out of range or a
 * NULL pointer. */
int64_t pcc_schedule_num_tiles(int64_t n, pcc_prec prec);
pcc_status pcc_schedule_tile_rect(int64_t n, pcc_prec prec, int64_t tile,
                                  int64_t *row0, int64_t *row1, int64_t *col0,
                                  int64_t *col1);

/* text of a status code (static storage) */
const char *pcc_status_string(pcc_status s);

#ifdef __cplusplus
}
#endif
#endif /* PCC_H */
