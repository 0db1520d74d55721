/*
 * oracle.c -- CPU oracle for CSR sparse matrix-vector multiplication computed
 * by speculative segmented sum (Liu & Vinter, "Speculative Segmented Sum for
 * Sparse Matrix-Vector Multiplication on Heterogeneous Processors").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the bench's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA path.  Everything is FP64 and plainly sequential per row or per tile,
 * compiled without floating-point contraction.
 *
 * Contents
 *   1. The plain definition y = A x (Sec. 2.1): a row loop, serial and with
 *      rows split over OpenMP threads (the paper's CPU row-block method,
 *      Sec. 4.3), plus a compensated reference (Dot2) and the per-row scale
 *      sum_k |val_k * x[col_k]| used by the tolerance.
 *   2. The index artefacts of the method, each from its definition:
 *      tile offsets (Sec. 3.2, rightmost match, by a linear merge rather than
 *      a binary search), raw segment descriptors (Sec. 3.2), dirty flags
 *      (Sec. 3.2 and Algorithm 1's empty-row test), segment counts.
 *   3. The paper's two stages simulated step by step (Algorithm 1 and the
 *      checking-prediction stage of Sec. 3.2), used to pin the worked
 *      example of Fig. 2 and to show that the method reproduces item 1.
 *
 * Readings of the paper (where it is silent or inconsistent):
 *   R1 boundaries past nnz are clamped to nnz; a tile holds
 *      len_t = b_{t+1} - b_t <= W*T entries.
 *   R2 the descriptor marks every row start inside the tile, including the
 *      start of row `stop` (Algorithm 1's descriptor loop stops one row short
 *      of it, which would merge row `stop` into row `stop-1`).
 *   R3 y is zero before the speculative stage, so a synchroniser entry for a
 *      row no earlier bunch wrote still yields the plain sum (Sec. 3.2).
 *   R4 on a dirty tile the transmitter is reset (Algorithm 1); the checking
 *      stage therefore ADDS that tile's last partial into y[stop] when row
 *      `stop` continues into the next tile, and moves the other partials.
 *   R5 rows before tile_offset[0] (leading empty rows) and rows emptied by
 *      the re-arrangement are exact zeros.
 *
 * Descriptor word layout (shared with nothing, restated by the CUDA side from
 * its own header): tile t owns ceil(W*T/32) uint32 words starting at word
 * t*ceil(W*T/32); bit k of the tile is bit (k % 32) of word k / 32.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* 1. the plain definition (Sec. 2.1): y_i = sum_{k in row i} val_k x[col_k] */

void oracle_spmv_rowloop(int32_t m, const int32_t *row_ptr, const int32_t *col,
                         const double *val, const double *x, double *y)
{
    for (int32_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            s += val[k] * x[col[k]];
        y[i] = s;
    }
}

/* same loop, rows split into contiguous blocks over OpenMP threads (the CPU
 * row-block method the paper benchmarks, Sec. 4.3).  Returns threads used. */
int oracle_spmv_rowloop_omp(int32_t m, const int32_t *row_ptr, const int32_t *col,
                            const double *val, const double *x, double *y, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    #pragma omp parallel num_threads(nthreads)
    {
        #pragma omp single
        used = omp_get_num_threads();
        #pragma omp for schedule(static)
        for (int32_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                s += val[k] * x[col[k]];
            y[i] = s;
        }
    }
#else
    (void)nthreads;
    oracle_spmv_rowloop(m, row_ptr, col, val, x, y);
#endif
    return used;
}

/* the plain definition restricted to the nonzeros [B, E): y_i = sum of
 * val_k x[col_k] over k in [row_ptr[i], row_ptr[i+1]) with B <= k < E (a row
 * with no entries there is 0).  Summing these over a partition of [0, nnz)
 * into ranges gives the row loop's y; it is what one shard of a product
 * split by tile ranges contributes to each row. */
void oracle_spmv_range(int32_t m, const int32_t *row_ptr, const int32_t *col,
                       const double *val, const double *x, int64_t B, int64_t E, double *y)
{
    for (int32_t i = 0; i < m; ++i) {
        int64_t lo = row_ptr[i] > B ? row_ptr[i] : B;
        int64_t hi = row_ptr[i + 1] < E ? row_ptr[i + 1] : E;
        double s = 0.0;
        for (int64_t k = lo; k < hi; ++k)
            s += val[k] * x[col[k]];
        y[i] = s;
    }
}

/* Error-free transformations: TwoSum (Knuth, TAOCP vol. 2) and TwoProduct by
 * fused multiply-add; Dot2 is Algorithm 5.3 of Ogita, Rump and Oishi,
 * "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005).  The result
 * is as accurate as if computed in twice the working precision and then
 * rounded.  scale_i = sum |val_k x[col_k]| (computed in plain FP64). */
static inline void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static inline void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

void oracle_spmv_dot2(int32_t m, const int32_t *row_ptr, const int32_t *col,
                      const double *val, const double *x, double *yref, double *scale)
{
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t i = 0; i < m; ++i) {
        double p = 0.0, s = 0.0, a = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double h, r, q;
            two_prod(val[k], x[col[k]], &h, &r);
            two_sum(p, h, &p, &q);
            s += q + r;
            a += fabs(val[k] * x[col[k]]);
        }
        yref[i] = p + s;
        if (scale) scale[i] = a;
    }
}

/* ------------------------------------------------------------------ */
/* 2. index artefacts from their definitions                          */

static inline int64_t bnd(int64_t t, int64_t L, int64_t nnz)
{
    int64_t b = t * L;
    return b < nnz ? b : nnz;                     /* R1 */
}

int64_t oracle_num_tiles(int64_t nnz, int64_t L)
{
    return (nnz + L - 1) / L;
}

/* tile_offset[t] = the largest r in [0, m] with row_ptr[r] <= b_t
 * (Sec. 3.2: the search returns the rightmost match).  Computed by one
 * forward merge of the boundaries with row_ptr. */
void oracle_tile_offsets(int32_t m, int32_t nnz, const int32_t *row_ptr, int32_t L,
                         int32_t *tile_offset)
{
    int64_t nt = oracle_num_tiles(nnz, L);
    int32_t r = 0;
    for (int64_t t = 0; t <= nt; ++t) {
        int64_t b = bnd(t, L, nnz);
        while (r < m && row_ptr[r + 1] <= b) ++r;
        tile_offset[t] = r;
    }
}

/* raw segment descriptor of every tile: bit k is set iff some row starts at
 * nnz position b_t + k (k < len_t).  Bit 0 is therefore set only when a row
 * really starts at the boundary; the method forces it afterwards (Sec. 3.2,
 * R2).  desc must hold ntiles*ceil(L/32) words. */
void oracle_descriptors(int32_t m, int32_t nnz, const int32_t *row_ptr, int32_t L,
                        const int32_t *tile_offset, uint32_t *desc)
{
    int64_t nt = oracle_num_tiles(nnz, L);
    int64_t wpt = (L + 31) / 32;
    memset(desc, 0, sizeof(uint32_t) * (size_t)(nt * wpt));
    for (int64_t t = 0; t < nt; ++t) {
        int64_t b = bnd(t, L, nnz), e = bnd(t + 1, L, nnz);
        uint32_t *w = desc + t * wpt;
        for (int32_t r = tile_offset[t]; r <= tile_offset[t + 1] && r <= m; ++r) {
            int64_t k = (int64_t)row_ptr[r] - b;
            if (k >= 0 && k < e - b)
                w[k / 32] |= 1u << (k % 32);
        }
    }
}

/* dirty[t] = 1 iff some row j in [start_t, stop_t) is empty (Sec. 3.2: an
 * empty row shows as two equal consecutive row pointers).  nseg[t] = number
 * of segments of tile t = number of row starts inside it, bit 0 forced. */
void oracle_tile_flags(int32_t m, int32_t nnz, const int32_t *row_ptr, int32_t L,
                       const int32_t *tile_offset, uint8_t *dirty, int32_t *nseg)
{
    int64_t nt = oracle_num_tiles(nnz, L);
    for (int64_t t = 0; t < nt; ++t) {
        int64_t b = bnd(t, L, nnz), e = bnd(t + 1, L, nnz);
        int32_t start = tile_offset[t], stop = tile_offset[t + 1];
        uint8_t d = 0;
        for (int32_t j = start; j < stop; ++j)
            if (row_ptr[j] == row_ptr[j + 1]) d = 1;
        int32_t cnt = 1;                                  /* position 0 */
        for (int32_t r = start; r <= stop && r <= m; ++r) {
            int64_t k = (int64_t)row_ptr[r] - b;
            if (k > 0 && k < e - b && (r == start || row_ptr[r] != row_ptr[r - 1]))
                ++cnt;
        }
        if (dirty) dirty[t] = d;
        if (nseg) nseg[t] = cnt;
    }
}

/* ------------------------------------------------------------------ */
/* 3. the paper's method simulated (Algorithm 1 and Sec. 3.2)          */

/* rightmost r in [0, m] with row_ptr[r] <= b (a plain binary search) */
static int32_t search_rightmost(int32_t m, const int32_t *row_ptr, int64_t b)
{
    int32_t lo = 0, hi = m;          /* invariant: row_ptr[lo] <= b */
    while (lo < hi) {
        int32_t mid = lo + (hi - lo + 1) / 2;
        if (row_ptr[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* Speculative execution stage for thread-bunches of T lanes, W entries per
 * lane and S tiles per bunch.  Outputs:
 *   y[m]                    speculative vector (zeroed first, R3)
 *   sync_idx/val[nbunches]  synchronizer, one entry per bunch
 *   spec_tile[ntiles]       speculator: ids of dirty tiles in bunch order
 *                           (the paper records <start, stop>; the tile id
 *                           identifies both and also its boundaries)
 *   returns dirty_counter, or -1 on allocation failure.
 * Per tile the steps follow the paper: search the S+1 boundaries, build the
 * descriptor and detect empty rows, form the products, take in the
 * transmitter, reduce segments (per lane: ts = position of its first head,
 * tc = number of heads), exclusive-scan tc into y_index, store partials, and
 * label a dirty tile. */
int64_t oracle_speculative_stage(int32_t m, int32_t nnz, const int32_t *row_ptr,
                                 const int32_t *col, const double *val, const double *x,
                                 int32_t T, int32_t W, int32_t S, double *y,
                                 int32_t *sync_idx, double *sync_val, int32_t *spec_tile)
{
    const int64_t L = (int64_t)W * T;
    const int64_t nb = (nnz + S * L - 1) / (S * L);
    uint8_t *desc = (uint8_t *)malloc((size_t)L);
    double *product = (double *)malloc(sizeof(double) * (size_t)L);
    double *partial = (double *)malloc(sizeof(double) * (size_t)L);
    int32_t *ts = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
    int32_t *tc = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
    int32_t *y_index = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
    int32_t *toff = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S + 1));
    int64_t *boundary = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S + 1));
    if (!desc || !product || !partial || !ts || !tc || !y_index || !toff || !boundary) {
        free(desc); free(product); free(partial); free(ts); free(tc); free(y_index);
        free(toff); free(boundary);
        return -1;
    }
    for (int32_t i = 0; i < m; ++i) y[i] = 0.0;                       /* R3 */
    int64_t dirty_counter = 0;
    for (int64_t tb = 0; tb < nb; ++tb) {
        /* positioning row indices of the S+1 tile boundaries */
        for (int32_t i = 0; i <= S; ++i) {
            boundary[i] = bnd(tb * S + i, L, nnz);
            toff[i] = search_rightmost(m, row_ptr, boundary[i]);
        }
        double transmitter = 0.0;
        for (int32_t i = 0; i < S; ++i) {
            if (boundary[i] >= nnz) break;                            /* R1 */
            const int64_t b = boundary[i], len = boundary[i + 1] - b;
            const int32_t start = toff[i], stop = toff[i + 1];
            /* segment descriptor and empty-row detection */
            memset(desc, 0, (size_t)L);
            int dirty = 0;
            for (int32_t j = start; j <= stop && j < m; ++j) {       /* R2 */
                if (row_ptr[j] != row_ptr[j + 1]) {
                    int64_t k = (int64_t)row_ptr[j] - b;
                    if (k >= 0 && k < len) desc[k] = 1;
                } else if (j < stop) {
                    dirty = 1;
                }
            }
            /* element-wise products (positions past len contribute nothing) */
            for (int64_t j = 0; j < L; ++j)
                product[j] = (j < len) ? x[col[b + j]] * val[b + j] : 0.0;
            /* transmitter from the previous tile */
            if (!desc[0]) {
                product[0] = product[0] + transmitter;
                desc[0] = 1;
            }
            /* segmented reduction over the W x T tile: lane j covers
             * positions [j*W, (j+1)*W); each head opens a segment whose sum
             * runs to the next head (possibly in a later lane).  Partials
             * are kept compactly: the lane's k-th head's sum is partial[
             * j*W + ts[j] + k] with ts[j] the slot of its first partial. */
            for (int32_t j = 0; j < T; ++j) {
                tc[j] = 0;
                ts[j] = 0;
                for (int32_t q = 0; q < W; ++q)
                    if (desc[(int64_t)j * W + q]) ++tc[j];
            }
            {
                int64_t pos = 0;
                while (pos < L) {
                    /* pos is a head: sum to the next head */
                    int64_t e = pos + 1;
                    while (e < L && !desc[e]) ++e;
                    double s = 0.0;
                    for (int64_t q = pos; q < e; ++q) s += product[q];
                    int32_t lane = (int32_t)(pos / W);
                    /* k-th head of this lane */
                    int32_t k = 0;
                    for (int64_t q = (int64_t)lane * W; q < pos; ++q) k += desc[q];
                    partial[(int64_t)lane * W + ts[lane] + k] = s;
                    pos = e;
                }
            }
            /* y_index = exclusive scan of tc */
            {
                int32_t acc = 0;
                for (int32_t j = 0; j < T; ++j) { y_index[j] = acc; acc += tc[j]; }
            }
            /* saving partial sums to y (first segment of the bunch goes to the
             * synchronizer) */
            for (int32_t j = 0; j < T; ++j) {
                for (int32_t k = 0; k < tc[j]; ++k) {
                    int64_t index = (int64_t)start + y_index[j] + k;
                    double v = partial[(int64_t)j * W + ts[j] + k];
                    if (index == toff[0]) {
                        sync_idx[tb] = (int32_t)index;
                        sync_val[tb] = v;
                    } else {
                        y[index] = v;
                    }
                    if (index == stop) transmitter = v;
                }
            }
            /* labeling a dirty tile */
            if (dirty) {
                spec_tile[dirty_counter++] = (int32_t)(tb * S + i);
                transmitter = 0.0;
            }
        }
    }
    free(desc); free(product); free(partial); free(ts); free(tc); free(y_index);
    free(toff); free(boundary);
    return dirty_counter;
}

/* Checking-prediction stage (Sec. 3.2): first the synchronisation (every
 * bunch adds its synchronizer value into y[idx]), then, if dirty_counter is
 * non-zero, the re-arrangement of each dirty tile's partials using row_ptr.
 * The s-th partial (s >= 1; stored at y[start + s]) belongs to the s-th row
 * of [start, stop] that has entries in the tile; rows of (start, stop)
 * without entries become zero (R5); a partial of row `stop` is added (R4). */
void oracle_checking_stage(int32_t m, int32_t nnz, const int32_t *row_ptr,
                           int32_t T, int32_t W, int32_t S, double *y,
                           const int32_t *sync_idx, const double *sync_val,
                           const int32_t *spec_tile, int64_t dirty_counter)
{
    const int64_t L = (int64_t)W * T;
    const int64_t nb = (nnz + S * L - 1) / (S * L);
    for (int64_t tb = 0; tb < nb; ++tb)
        y[sync_idx[tb]] = y[sync_idx[tb]] + sync_val[tb];
    for (int64_t d = 0; d < dirty_counter; ++d) {
        int64_t t = spec_tile[d];
        int64_t b = bnd(t, L, nnz), e = bnd(t + 1, L, nnz);
        int32_t start = search_rightmost(m, row_ptr, b);
        int32_t stop = search_rightmost(m, row_ptr, e);
        /* the rows that own segments, in order */
        int64_t cap = (int64_t)stop - start + 1;
        int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
        double *moved = (double *)malloc(sizeof(double) * (size_t)cap);
        if (!rows || !moved) { free(rows); free(moved); return; }
        int64_t ns = 0;
        for (int32_t r = start; r <= stop && r < m; ++r)
            if (row_ptr[r] < row_ptr[r + 1] && row_ptr[r] < e)
                rows[ns++] = r;
        for (int64_t s = 1; s < ns; ++s) moved[s] = y[start + s];
        for (int32_t r = start + 1; r < stop; ++r) y[r] = 0.0;
        for (int64_t s = 1; s < ns; ++s) {
            if (rows[s] == stop) y[stop] = y[stop] + moved[s];
            else y[rows[s]] = moved[s];
        }
        free(rows);
        free(moved);
    }
}
