/*
 * ssspmv.h -- C ABI of a GB300 (sm_103a) CSR sparse matrix-vector multiply
 * computed as a speculative segmented sum (Liu & Vinter, "Speculative
 * Segmented Sum for Sparse Matrix-Vector Multiplication on Heterogeneous
 * Processors").
 *
 * The operation is y = A x for an m x n matrix A in CSR form (Sec. 2.1):
 *   row_ptr[m+1], col_idx[nnz], val[nnz], x[n] -> y[m]
 * with y overwritten (no alpha/beta) and every row written, empty rows as 0.
 *
 * The nonzeros are cut into tiles of L = 32*W entries (Sec. 3.1: T = 32 lanes
 * of a warp, W entries per lane); a warp ("thread-bunch") processes S
 * consecutive tiles.  Three kernels run on the caller's stream:
 *   (a) partition: tile_offset[t] = the largest r with row_ptr[r] <= t*L
 *       (Sec. 3.2 and Algorithm 1: binary search, rightmost match);
 *   (b) segmented sum: per tile, the row-start descriptor is built on chip
 *       from row_ptr, products val*x[col] are reduced per segment, and each
 *       segment s is stored speculatively to y[tile_offset[t] + s]; the first
 *       segment of each bunch goes to a synchronizer record (Sec. 3.2,
 *       Algorithm 1);
 *   (c) calibration: synchronizer records are summed into their rows, the
 *       partials of tiles holding empty rows ("dirty" tiles) are moved to
 *       their true rows, and empty rows are zeroed (Sec. 3.2, checking
 *       prediction, and Algorithm 1's synchronization step, here on the GPU).
 *
 * Conventions for every entry point below:
 *   - Array pointers are DEVICE pointers unless the name says host, owned by
 *     the caller; the library never frees caller memory.  Calls are
 *     asynchronous on `stream` (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream); inputs must stay valid until it completes.
 *   - Indices are 0-based int32 (the paper's idx_type, Sec. 4.3); nnz must fit
 *     in int32.  Column order inside a row is free; duplicates are summed.
 *   - `val` and `col_idx` must be 16-byte aligned (they are streamed by bulk
 *     asynchronous copies); x and y need only natural alignment.
 *   - Column indices must lie in [0, n); an out-of-range column is undefined
 *     behaviour (call ssspmv_validate_csr first for untrusted input).
 *   - Return value: SSSPMV_OK (0) or a negative code; nothing is launched
 *     when a host-side check fails.  No C++ exception crosses the ABI.
 *   - The same input gives bit-identical y on every run (no floating-point
 *     atomics; all reductions have a fixed order).
 */
#ifndef SSSPMV_H
#define SSSPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SSSPMV_OK            0
#define SSSPMV_EINVAL       -1  /* bad scalar, null pointer with size > 0, misalignment, bad opts */
#define SSSPMV_EWORKSPACE   -2  /* workspace NULL or smaller than ssspmv_workspace_bytes() */
#define SSSPMV_ECUDA        -3  /* a CUDA call failed; see ssspmv_last_cuda_error() */
#define SSSPMV_EDEVICE      -4  /* a kernel reported an inconsistency or a timed-out wait */
#define SSSPMV_EUNSUPPORTED -5  /* tile shape not compiled into the library */
#define SSSPMV_ETOOLARGE    -6  /* problem needs more scratch than ssspmv_csr_f64_noalloc has */

/* Largest m and nnz accepted (larger values return SSSPMV_EINVAL): the
 * kernels index rows and entries in 32-bit integers with 256 of headroom. */
#define SSSPMV_MAX_DIM (2147483647 - 256)

/* Device error bits written by the kernels into the workspace (read with
 * ssspmv_device_status). */
#define SSSPMV_DEV_TIMEOUT   1u  /* a bounded wait on a bulk copy gave up */
#define SSSPMV_DEV_RANGE     2u  /* a computed row index fell outside [0, m) */
#define SSSPMV_DEV_CALIB     4u  /* calibration found a segment count that does not match row_ptr */
#define SSSPMV_DEV_BATCH     8u  /* a batch descriptor was invalid (that matrix was skipped) or
                                    the batch exceeded the capacity its workspace was sized for
                                    (nothing was computed) */

/* Storing the partial sums of tiles that hold empty rows ("dirty" tiles):
 *  SPECULATIVE  the paper's method: kernel (b) stores every segment at its
 *               speculative row tile_offset[t] + s and kernel (c) moves the
 *               partials of dirty tiles to their rows and zeroes empty rows
 *               (Sec. 3.2, checking prediction).  The default.
 *  EXACT        kernel (b) resolves dirty tiles on chip: it already reads the
 *               tile's row pointers, so it stores each partial at the row that
 *               starts at the segment's head and zeroes the empty rows itself;
 *               kernel (c) only finishes the synchronizer sums.  Same y. */
#define SSSPMV_VARIANT_DEFAULT     0
#define SSSPMV_VARIANT_SPECULATIVE 1
#define SSSPMV_VARIANT_EXACT       2
/*  ROWS         not the paper's method but the row-parallel CSR kernels it
 *               compares against (Sec. 2.1, 4.3), offered as a class for the
 *               variant selector: a group of opts->W lanes per row (1 = the
 *               scalar kernel, 2..32 powers of two = the vector kernel; 0 =
 *               from the mean row length).  No partition and no calibration;
 *               FP64 single calls only (the FP32/BF16, plan and batched entry
 *               points return SSSPMV_EUNSUPPORTED). */
#define SSSPMV_VARIANT_ROWS        3

/* Tile and launch parameters (Sec. 3.1, Table 3).  Zero-initialise and set
 * only what you need; a NULL opts pointer means all defaults. */
typedef struct ssspmv_opts {
    int32_t W;         /* entries per lane (odd, see ssspmv_supported_w); L = 32*W.
                          0 = the shortest compiled tile (BF16 values: 27 when rows
                          hold 20 entries or more on average).  With SSSPMV_VARIANT_ROWS:
                          lanes per row (see there) */
    int32_t S;         /* tiles per thread-bunch (warp); 0 = 4, or fewer for matrices of
                          under 98,304 tiles (ceil(ntiles / 32768)).  Each warp of a
                          persistent grid first takes an even contiguous share of
                          3/4 of the bunches, then single bunches from a counter */
    int32_t block_warps; /* warps per block of the segmented-sum kernel (one block
                          per SM).  0 = automatic: all that fit in shared memory
                          when the mean row length nnz/m is at least 20, else as
                          many as leave about 56 KB of L1 for the x gathers;
                          values above the most that fit are lowered to it */
    int32_t variant;   /* SSSPMV_VARIANT_*: how tiles holding empty rows are stored */
    void   *timer;     /* optional ssspmv_timer*: the call records its kernel
                          boundaries into the timer's next slot; NULL = none */
} ssspmv_opts;

/* Stage timing with events owned by this library (events created by another
 * CUDA runtime instance in the process cannot be recorded from here).  A
 * timer holds `capacity` slots; every call given the timer in opts->timer
 * records 4 events on its stream into the next free slot (before kernel (a),
 * before (b), before (c), after (c)); calls beyond capacity are not timed.
 * Not thread safe: one timer per stream. */
typedef struct ssspmv_timer ssspmv_timer;
int ssspmv_timer_create(int32_t capacity, ssspmv_timer **out);
void ssspmv_timer_destroy(ssspmv_timer *t);
/* forget recorded slots (the events are reused) */
void ssspmv_timer_reset(ssspmv_timer *t);
/* waits for the recorded events and writes, for slot i < *count (at most cap
 * slots): ms[4i] = kernel (a), ms[4i+1] = kernel (b), ms[4i+2] = kernel (c),
 * ms[4i+3] = the whole call, in milliseconds */
int ssspmv_timer_read(ssspmv_timer *t, float *ms, int32_t cap, int32_t *count);

/* The tile shape and bunch count a call with these arguments would use.
 * val_bytes = sizeof the stored value type: 8 (FP64), 4 (FP32) or 2 (BF16).  Any output pointer
 * may be NULL.  Returns SSSPMV_OK or SSSPMV_EINVAL/EUNSUPPORTED. */
int ssspmv_plan_shape(int32_t m, int32_t nnz, int32_t val_bytes, const ssspmv_opts *opts,
                      int32_t *W, int32_t *L, int32_t *S, int64_t *ntiles, int64_t *nbunches);

/* Bytes of device workspace needed by a call with these arguments
 * (tile offsets, per-tile info, synchronizer records; the paper's
 * pre-allocated containers, Sec. 3.3).  Returns 0 on invalid arguments. */
size_t ssspmv_workspace_bytes(int32_t m, int32_t nnz, int32_t val_bytes, const ssspmv_opts *opts);

/* y = A x in FP64 (val, x, y double).  workspace: device buffer of at least
 * ssspmv_workspace_bytes(m, nnz, 8, opts) bytes, 256-byte aligned, not used
 * by another call in flight -- or NULL (ws_bytes ignored) for a buffer the
 * library owns, cached per (device, stream) and grown stream-ordered with
 * cudaMallocAsync on `stream` when a call needs more (see
 * ssspmv_cached_workspace).  Kernels: (a), (b), (c) above. */
int ssspmv_csr_f64(int32_t m, int32_t n, int32_t nnz,
                   const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                   const double *x, double *y,
                   const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream);

/* y = A x with FP32 val, x and y.  Products are split exactly (TwoProduct)
 * and summed with TwoSum into an unevaluated FP32 pair per segment; the
 * synchronizer sums of rows crossing bunches are finished in FP64.
 * workspace: ssspmv_workspace_bytes(m, nnz, 4, opts) bytes. */
int ssspmv_csr_f32(int32_t m, int32_t n, int32_t nnz,
                   const int32_t *row_ptr, const int32_t *col_idx, const float *val,
                   const float *x, float *y,
                   const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream);

/* y = A x with BF16 val (raw bfloat16 bits), FP32 x and y, accumulated as in
 * ssspmv_csr_f32.  workspace: ssspmv_workspace_bytes(m, nnz, 2, opts) bytes. */
int ssspmv_csr_bf16f32(int32_t m, int32_t n, int32_t nnz,
                       const int32_t *row_ptr, const int32_t *col_idx, const uint16_t *val,
                       const float *x, float *y,
                       const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream);

/* y = alpha A x + beta y in FP64 (the iterative-solver form; the paper computes
 * y = A x only).  Same arguments and contract as ssspmv_csr_f64 plus the two
 * scalars; y is read only where beta != 0 (so with beta == 0 it may hold
 * anything, NaN included).  The partials of tiles with empty rows are always
 * stored at their true rows (SSSPMV_VARIANT_EXACT, whatever opts->variant
 * says, except SSSPMV_VARIANT_ROWS), because a speculative store would
 * overwrite a row of y before its old value is read.  Each row's result is
 * fma(beta, y_old, alpha * (A x)_row). */
int ssspmv_csr_f64_axpby(int32_t m, int32_t n, int32_t nnz,
                         const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                         const double *x, double *y, double alpha, double beta,
                         const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream);

/* The library-owned workspace of the current device and `stream` (the one
 * calls with workspace == NULL use), e.g. for ssspmv_device_status.  Returns
 * SSSPMV_EWORKSPACE (and NULL, 0) if no call on that stream has made one yet.
 * ssspmv_release_workspaces frees every cached buffer (cudaFree: waits for the
 * work still using them); call it when no call is in flight. */
int ssspmv_cached_workspace(void *stream, void **ptr, size_t *bytes);
void ssspmv_release_workspaces(void);

/* Partition reuse for iterative solvers (one sparsity pattern, many
 * products).  The paper has no plan -- its method needs no preprocessing
 * (Sec. 1), and the single calls above are what the headline numbers time --
 * but kernel (a) depends on row_ptr alone, so a plan runs it once:
 *   ssspmv_plan_create  checks the arguments, resolves the tile shape for the
 *     stored value type (val_bytes 8, 4 or 2; opts as for the single calls,
 *     opts->timer must be NULL), takes `workspace` (NULL: the plan allocates
 *     one with cudaMalloc and owns it) and launches kernel (a) on `stream`.
 *     row_ptr stays the caller's: it must remain valid and unchanged while
 *     the plan lives (kernel (b) reads it on every execution).
 *   ssspmv_plan_execute  y = A x with the plan's partition: kernels (b) and
 *     (c) on `stream`, for col_idx/val/x/y of the plan's value type (double,
 *     float, or bf16 val with float x and y).  It allocates nothing; `timer`
 *     (nullable ssspmv_timer*) records it, its kernel (a) slot then timing the
 *     reset of the error word.  Executions of one plan share its workspace:
 *     order them on one stream.  Must run on the plan's device.
 *   ssspmv_plan_workspace  the plan's workspace (for ssspmv_device_status).
 *   ssspmv_plan_destroy  frees what the plan owns (cudaFree: waits for the
 *     device). */
typedef struct ssspmv_plan ssspmv_plan;
int ssspmv_plan_create(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                       int32_t val_bytes, const ssspmv_opts *opts, void *workspace,
                       size_t ws_bytes, void *stream, ssspmv_plan **out);
int ssspmv_plan_execute(ssspmv_plan *plan, const int32_t *col_idx, const void *val,
                        const void *x, void *y, void *timer, void *stream);
int ssspmv_plan_workspace(const ssspmv_plan *plan, void **ptr, size_t *bytes);
/* y = alpha A x + beta y with the plan's partition (FP64 plans only, else
 * SSSPMV_EUNSUPPORTED); exact stores, as for ssspmv_csr_f64_axpby. */
int ssspmv_plan_execute_axpby(ssspmv_plan *plan, const int32_t *col_idx, const void *val,
                              const void *x, void *y, double alpha, double beta, void *timer,
                              void *stream);
void ssspmv_plan_destroy(ssspmv_plan *plan);

/* Batched FP32 products y_i = A_i x_i for `count` matrices of any sizes in
 * one pass: a set-up kernel, kernel (a) over every matrix, ONE persistent
 * launch of kernel (b) over every bunch of every matrix (bunches never cross
 * matrices) and kernel (c) over all of them -- four launches whatever the
 * count, no host synchronisation and no allocation, so the call can be
 * captured in a CUDA graph.  The paper runs one matrix at a time; batching is
 * this library's addition.
 *   mats       DEVICE array of `count` descriptors, 8-byte aligned; each
 *              describes one matrix exactly as the single FP32 call takes it
 *              (float val, x, y; col_idx and val 16-byte aligned; reserved 0).
 *              An invalid descriptor is skipped (its y untouched) and sets
 *              SSSPMV_DEV_BATCH in the workspace's error word.
 *   total_nnz  an upper bound of the sum of the matrices' nnz: it sizes the
 *              workspace (ssspmv_batched_workspace_bytes with the same count,
 *              total_nnz and opts).  A batch that turns out larger computes
 *              nothing and sets SSSPMV_DEV_BATCH.
 *   opts       as for the single calls (one tile shape W and bunch size S for
 *              the whole batch; opts->timer records the four launches as
 *              set-up+(a), (b), (c)).
 * Results equal the single FP32 call's bit for bit for every matrix. */
typedef struct ssspmv_csr_desc {
    int32_t m, n, nnz;
    int32_t reserved;            /* must be 0 */
    const int32_t *row_ptr;      /* [m+1] */
    const int32_t *col_idx;      /* [nnz] */
    const void *val;             /* [nnz] float */
    const void *x;               /* [n] float */
    void *y;                     /* [m] float, written */
} ssspmv_csr_desc;               /* 56 bytes */
size_t ssspmv_batched_workspace_bytes(int32_t count, int64_t total_nnz, int32_t val_bytes,
                                      const ssspmv_opts *opts);
int ssspmv_csr_batched_f32(int32_t count, const ssspmv_csr_desc *mats, int64_t total_nnz,
                           const ssspmv_opts *opts, void *workspace, size_t ws_bytes,
                           void *stream);

/* Learned variant selector (not in the paper; it only chooses among the
 * kernels above and never changes their arithmetic).
 *   ssspmv_features  16 statistics of row_ptr alone, each of order one, into
 *     device float[16] (one pass over the rows twice, then one thread):
 *     log2 m, log2 nnz, log2 mean row length, coefficient of variation of the
 *     lengths, log2 max length, fractions of empty rows, of rows <= 4, of
 *     rows >= 2x the mean, of entries in rows > 1024, median / 90th / 99th
 *     percentile of log2 lengths, fraction of neighbours differing > 2x,
 *     log2 rows per 480-entry tile, fraction of empty rows after an empty
 *     row, fraction of entries in rows >= 32x the mean.  `scratch`: device
 *     memory of ssspmv_features_scratch_bytes().
 *   A perceptron F -> H1 -> H2 -> K (ReLU, ReLU, linear), FP32, parameters in
 *   one device array (ssspmv_mlp_param_count floats: W1[H1][F], b1[H1],
 *   W2[H2][H1], b2[H2], W3[K][H2], b3[K]), batch X[B][F] row-major; `scratch`
 *   holds ssspmv_mlp_scratch_floats(B, ...) floats.
 *   ssspmv_mlp_forward   out[B][K] (NULL: leave it in scratch).
 *   ssspmv_mlp_backward  forward, then the gradient of the mean squared error
 *     against target[B][K] (NaN targets count as 0 error) into grad (same
 *     layout as params) and the loss into *loss (device float, may be NULL).
 *   ssspmv_mlp_adam      one Adam step (Kingma & Ba) with L2 weight decay.
 *   ssspmv_mlp_select    cls[b] = argmin over k of the predicted out[b][k].
 * All asynchronous on `stream`; deterministic (fixed reduction orders). */
size_t ssspmv_features_scratch_bytes(void);
int ssspmv_features(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr, float *features,
                    void *scratch, void *stream);
int64_t ssspmv_mlp_param_count(int32_t F, int32_t H1, int32_t H2, int32_t K);
size_t ssspmv_mlp_scratch_floats(int32_t B, int32_t F, int32_t H1, int32_t H2, int32_t K);
int ssspmv_mlp_forward(const float *params, const float *X, int32_t B, int32_t F, int32_t H1,
                       int32_t H2, int32_t K, float *scratch, float *out, void *stream);
int ssspmv_mlp_backward(const float *params, const float *X, const float *target, int32_t B,
                        int32_t F, int32_t H1, int32_t H2, int32_t K, float *scratch, float *grad,
                        float *loss, void *stream);
int ssspmv_mlp_adam(float *params, const float *grad, float *m1, float *m2, int64_t n, float lr,
                    float beta1, float beta2, float eps, float weight_decay, int32_t step,
                    void *stream);
int ssspmv_mlp_select(const float *params, const float *X, int32_t B, int32_t F, int32_t H1,
                      int32_t H2, int32_t K, float *scratch, int32_t *cls, void *stream);

/* Allocation-free FP64 product.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code handed
 * only device pointers for A, x and y with no allocator of its own (a plug-in
 * inside another application's solver loop whose memory belongs to that
 * application), or code that must not call cudaMalloc/cudaFree on its hot
 * path because those calls can synchronise the device and stall other
 * streams.  Same arguments and result as ssspmv_csr_f64, without the
 * workspace: the workspace lives in a fixed device array of
 * SSSPMV_NOALLOC_SCRATCH_BYTES owned by the library, held by every GPU that
 * loads the library until the process exits.  Problems whose
 * ssspmv_workspace_bytes(m, nnz, 8, opts) exceeds it are rejected with
 * SSSPMV_ETOOLARGE before anything runs (8 MiB covers about 466,000 tiles
 * with the automatic bunch count -- 12 bytes of tile data per tile plus 24
 * bytes of synchronizer record per bunch of 4 -- i.e. nnz up to 223,671,840
 * at W = 15); options the other calls reject are rejected with the same
 * code.  All calls on a device share the array and it keeps the last call's
 * contents: each call clears its 16-byte header (error word, bunch ticket,
 * dirty-tile count, schedule flag) with cudaMemsetAsync on `stream`, and the
 * kernels write every other entry before reading it.  Calls that overlap on the GPU race
 * on the array -- order them on one stream.  The first call on a device
 * looks up the array's address (cudaGetSymbolAddress) with that device
 * current and caches it; make it before any stream capture begins.
 * `stream` must belong to the current device (else SSSPMV_EINVAL).  A
 * cudaDeviceReset invalidates the cached address: do not call this entry
 * point again in that process.  No call allocates device memory. */
#define SSSPMV_NOALLOC_SCRATCH_BYTES (8u << 20)
int ssspmv_csr_f64_noalloc(int32_t m, int32_t n, int32_t nnz,
                           const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                           const double *x, double *y, const ssspmv_opts *opts, void *stream);

/* One product split across devices by tile ranges (not in the paper, which
 * runs on one processor; the combination is its synchronization step of
 * Sec. 3.2 and Algorithm 1 one level up, between shards instead of
 * thread-bunches).  Shard g takes the tiles [t0, t1) of the whole matrix's
 * tiling (the same opts, hence the same tile length L, on every shard),
 * i.e. the nonzeros [B, E) = [min(t0 L, nnz), min(t1 L, nnz)).  Its rows
 * are r_first = the largest r with row_ptr[r] <= B and r_last = the largest r
 * with row_ptr[r] <= E (m for the shard that ends the matrix):
 *   - rows strictly between them lie inside [B, E): the shard writes their
 *     final y (empty rows 0);
 *   - rows r_first and r_last are cut: the shard writes its partial sums of
 *     them into y and into `seam`, and the sum over all shards' partials of
 *     such a row is its y (ssspmv_seam_merge);
 *   - the shard with t0 = 0 also zeroes the leading empty rows [0, r_first).
 * Shards share nothing on the device; the seam records (32 bytes each) are
 * the only exchange.  Their tiles are the unsplit product's tiles, so each
 * tile's arithmetic is the same as in ssspmv_csr_f64.
 *   ssspmv_range_bounds   r_first and r_last of [t0, t1) from the device
 *     row_ptr (a search kernel; allocates 8 bytes stream-ordered and
 *     synchronises `stream`).  0 <= t0 <= t1 <= ntiles (ssspmv_plan_shape).
 *   ssspmv_range_workspace_bytes  device workspace of the range call
 *     (the shard's shifted row pointers plus the workspace of its rows).
 *   ssspmv_csr_f64_range  the shard's product on `stream`: kernels (a), (b),
 *     (c) on rows [r_first, r_last] (r_last < m) or [r_first, m), with
 *     row_ptr shifted by B and clamped to [0, E - B], col_idx and val read
 *     from entry B on; then `seam` (DEVICE pointer) receives {r_first, its
 *     partial} and {r_last, its partial} (row -1 where there is no second
 *     cut row) and status 0, or SSSPMV_DEV_RANGE if r_first/r_last do not
 *     match row_ptr (then y is not the product).  opts->timer must be NULL;
 *     ROWS is not supported.  Arrays as for ssspmv_csr_f64 (x whole).
 *   ssspmv_seam_merge  HOST records of `shards` shards in shard order ->
 *     the cut rows and their final values (each the sum of that row's
 *     partials in shard order, so deterministic); rows/vals (host, up to
 *     2*shards entries, may be NULL to count) and *count.  Returns
 *     SSSPMV_EDEVICE if a record has a non-zero status, SSSPMV_EINVAL if the
 *     records are out of order.  The caller then stores vals into y[rows]. */
typedef struct ssspmv_seam {
    int32_t row[2];   /* rows cut at the shard's start and end; -1: none */
    int32_t status;   /* 0, or SSSPMV_DEV_RANGE (bounds do not match row_ptr) */
    int32_t reserved;
    double val[2];    /* the shard's partial sums of those rows */
} ssspmv_seam;        /* 32 bytes */
int ssspmv_range_bounds(int32_t m, int32_t nnz, const int32_t *row_ptr, const ssspmv_opts *opts,
                        int64_t t0, int64_t t1, int32_t *r_first, int32_t *r_last, void *stream);
size_t ssspmv_range_workspace_bytes(int32_t m, int32_t nnz, int64_t t0, int64_t t1,
                                    int32_t r_first, int32_t r_last, const ssspmv_opts *opts);
int ssspmv_csr_f64_range(int32_t m, int32_t n, int32_t nnz,
                         const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                         const double *x, double *y, int64_t t0, int64_t t1,
                         int32_t r_first, int32_t r_last, ssspmv_seam *seam,
                         const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream);
int ssspmv_seam_merge(int32_t shards, const ssspmv_seam *seams, int32_t *rows, double *vals,
                      int32_t *count);

/* The same product with HOST arrays (pageable or pinned): copies row_ptr,
 * col_idx, val and x into `dev_buffer` (device memory of at least
 * ssspmv_host_buffer_bytes() bytes), runs ssspmv_csr_f64 on `stream`, copies
 * y back to host_y and synchronises the stream before returning. */
size_t ssspmv_host_buffer_bytes(int32_t m, int32_t n, int32_t nnz, const ssspmv_opts *opts);
int ssspmv_csr_f64_host(int32_t m, int32_t n, int32_t nnz,
                        const int32_t *host_row_ptr, const int32_t *host_col_idx,
                        const double *host_val, const double *host_x, double *host_y,
                        const ssspmv_opts *opts, void *dev_buffer, size_t dev_bytes,
                        void *stream);

/* FP64 product that also exports the method's index artefacts for checking
 * against an independent derivation (any output may be NULL):
 *   tile_offset[ntiles+1]   kernel (a)'s partition (Sec. 3.2)
 *   desc[ntiles*W]          raw segment descriptor words of kernel (b): bit k
 *                           of tile t is bit k%32 of word t*W + k/32, set iff a
 *                           row starts at entry t*L + k (bit 0 NOT forced)
 *   tile_info[ntiles]       bit 31 = dirty (an empty row in [start, stop)),
 *                           bit 30 = dirty and resolved in kernel (b) (EXACT),
 *                           bits 0..29 = number of segments of the tile
 *   sync_idx[nbunches]      synchronizer row of each bunch (= tile_offset[w*S])
 *   y_spec[m]               y after kernel (b), before calibration (entries
 *                           kernel (b) does not write are left as y held them)
 * Synchronises the stream and returns SSSPMV_EDEVICE if a kernel flagged an
 * error. */
int ssspmv_csr_f64_debug(int32_t m, int32_t n, int32_t nnz,
                         const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                         const double *x, double *y,
                         const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream,
                         int32_t *tile_offset, uint32_t *desc, uint32_t *tile_info,
                         int32_t *sync_idx, double *y_spec);

/* Checks a CSR structure on the device: row_ptr[0] == 0, row_ptr[m] == nnz,
 * row_ptr non-decreasing, 0 <= col_idx < n.  `scratch` is 16 bytes of device
 * memory.  Synchronises the stream.  Returns SSSPMV_OK or SSSPMV_EINVAL. */
int ssspmv_validate_csr(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, void *scratch, void *stream);

/* Device error bits (SSSPMV_DEV_*) accumulated in this workspace since it was
 * last cleared; synchronises the stream.  clear != 0 resets them. */
int ssspmv_device_status(void *workspace, size_t ws_bytes, void *stream, int clear,
                         uint32_t *bits);

/* Odd W values compiled into the library, written to out[0..*count). */
int ssspmv_supported_w(int32_t *out, int32_t cap, int32_t *count);

const char *ssspmv_strerror(int code);
int ssspmv_last_cuda_error(void);     /* cudaError_t of the last failed CUDA call */
int ssspmv_version(void);             /* major*10000 + minor*100 + patch */

#ifdef __cplusplus
}
#endif

#endif /* SSSPMV_H */
