/*
 * synth.c -- seeded, deterministic synthetic CSR inputs.
 *
 * This module only manufactures inputs (row pointers, column indices, values
 * and dense vectors).  It holds none of the sparse matrix-vector arithmetic:
 * both the CPU oracle and the CUDA path consume what it writes, and neither
 * shares any other code.
 *
 * Randomness is counter based, so every output element is a pure function of
 * (seed, stream, counter) and the result is identical on any machine, thread
 * count or schedule.  The generator is the SplitMix64 construction of Steele,
 * Lea and Flood ("Fast splittable pseudorandom number generators", OOPSLA
 * 2014): a Weyl sequence with increment 0x9E3779B97F4A7C15 passed through the
 * 64-bit finalising mixer (Stafford's "variant 13").  Here the Weyl state is
 * addressed directly by the counter instead of being advanced.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define WEYL 0x9E3779B97F4A7C15ULL

enum {
    ST_LEN = 1,      /* row lengths */
    ST_EMPTY = 2,    /* choice of rows forced empty */
    ST_COL = 3,      /* column sampling */
    ST_VAL = 4,      /* matrix values */
    ST_VEC = 5,      /* dense vectors (caller passes its own stream too) */
    ST_RMAT = 6,     /* R-MAT quadrant draws */
    ST_INJROW = 7,   /* which row receives the injected long row */
    ST_INJCOL = 8,   /* columns of the injected long row */
};

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t synth_u64(uint64_t seed, uint64_t stream, uint64_t i)
{
    uint64_t key = mix64(seed * WEYL + mix64(stream + WEYL));
    return mix64(key + (i + 1) * WEYL);
}

/* uniform in [0, 1) with 53 random bits */
double synth_unit(uint64_t seed, uint64_t stream, uint64_t i)
{
    return (double)(synth_u64(seed, stream, i) >> 11) * 0x1.0p-53;
}

/* uniform in [-1, 1) */
static inline double sym(uint64_t seed, uint64_t stream, uint64_t i)
{
    return 2.0 * synth_unit(seed, stream, i) - 1.0;
}

/* unbiased-enough integer in [0, k) for k << 2^64 (multiply-shift) */
static inline uint64_t below(uint64_t seed, uint64_t stream, uint64_t i, uint64_t k)
{
    return (uint64_t)(((unsigned __int128)synth_u64(seed, stream, i) * k) >> 64);
}

/* ------------------------------------------------------------------ */
/* dense vector, entries uniform in [-1, 1)                            */
void synth_sym_vector(int64_t n, uint64_t seed, uint64_t stream, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        out[i] = sym(seed, ST_VEC * 1000003ULL + stream, (uint64_t)i);
}

/* ------------------------------------------------------------------ */
/* k distinct sorted integers from [0, n), drawn with counters          */
/* base..base+n-1 (selection sampling, Knuth TAOCP vol. 2, Alg. 3.4.2S) */
static void select_sorted(int64_t n, int64_t k, uint64_t seed, uint64_t stream,
                          uint64_t base, int32_t *out)
{
    int64_t got = 0;
    for (int64_t c = 0; c < n && got < k; ++c) {
        double u = synth_unit(seed, stream, base + (uint64_t)c);
        if ((double)(n - c) * u < (double)(k - got))
            out[got++] = (int32_t)c;
    }
}

/* k distinct sorted integers from [0, n) by Floyd's algorithm (Bentley,
 * "Programming Pearls" column 13) with a sorted array as the set.  O(k^2),
 * used for short rows. */
static void floyd_sorted(int64_t n, int64_t k, uint64_t seed, uint64_t stream,
                         uint64_t base, int32_t *out)
{
    int64_t cnt = 0;
    for (int64_t j = n - k; j < n; ++j) {
        int64_t t = (int64_t)below(seed, stream, base + (uint64_t)(j - (n - k)),
                                   (uint64_t)(j + 1));
        /* binary search for t */
        int64_t lo = 0, hi = cnt;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (out[mid] < t) lo = mid + 1; else hi = mid;
        }
        int64_t v = (lo < cnt && out[lo] == t) ? j : t;
        if (v != t) {  /* insert j: it is larger than every element so far */
            out[cnt++] = (int32_t)v;
        } else {
            memmove(out + lo + 1, out + lo, (size_t)(cnt - lo) * sizeof(int32_t));
            out[lo] = (int32_t)v;
            ++cnt;
        }
    }
}

static void distinct_sorted(int64_t n, int64_t k, uint64_t seed, uint64_t stream,
                            uint64_t base, int32_t *out)
{
    if (k <= 0) return;
    if (k * 8 > n || k > 512)
        select_sorted(n, k, seed, stream, base, out);
    else
        floyd_sorted(n, k, seed, stream, base, out);
}

/* ------------------------------------------------------------------ */
/* Uniform-length rows: length ~ U{0..maxlen}; then round(empty_frac*m)  */
/* rows (a seeded partial Fisher-Yates choice) are forced empty.         */
/* Writes row_ptr[m+1]; returns nnz.                                    */
int64_t synth_uniform_rows_ptr(int32_t m, int32_t maxlen, double empty_frac,
                               uint64_t seed, int32_t *row_ptr)
{
    int32_t *len = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!len || !perm) { free(len); free(perm); return -1; }
    for (int32_t r = 0; r < m; ++r) {
        len[r] = (int32_t)below(seed, ST_LEN, (uint64_t)r, (uint64_t)maxlen + 1);
        perm[r] = r;
    }
    int64_t k = (int64_t)llround(empty_frac * (double)m);
    if (k > m) k = m;
    for (int64_t i = 0; i < k; ++i) {
        int64_t j = i + (int64_t)below(seed, ST_EMPTY, (uint64_t)i, (uint64_t)(m - i));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        len[perm[i]] = 0;
    }
    int64_t acc = 0;
    row_ptr[0] = 0;
    for (int32_t r = 0; r < m; ++r) {
        acc += len[r];
        row_ptr[r + 1] = (int32_t)acc;
    }
    free(len);
    free(perm);
    return acc;
}

/* Fill sorted distinct columns (uniform over [0, n)) and values U[-1,1)  */
/* for a row_ptr produced by any generator.                             */
void synth_fill_uniform(int32_t m, int32_t n, const int32_t *row_ptr, uint64_t seed,
                        int32_t *col, double *val)
{
    #pragma omp parallel for schedule(dynamic, 64)
    for (int32_t r = 0; r < m; ++r) {
        int64_t b = row_ptr[r], e = row_ptr[r + 1];
        distinct_sorted(n, e - b, seed, ST_COL, (uint64_t)r * (uint64_t)n, col + b);
    }
    int64_t nnz = row_ptr[m];
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nnz; ++k)
        val[k] = sym(seed, ST_VAL, (uint64_t)k);
}

/* ------------------------------------------------------------------ */
/* 27-point stencil on an nx*ny*nz grid, lexicographic rows (x fastest), */
/* sorted columns.  Diagonal 26.0, off-diagonals -1.0 + U[-0.01, 0.01). */
/* col/val may be NULL to count only.  Returns nnz.                     */
static inline int32_t span3(int32_t i, int32_t n) { return 1 + (i > 0) + (i < n - 1); }

int64_t synth_stencil27(int32_t nx, int32_t ny, int32_t nz, uint64_t seed,
                        int32_t *row_ptr, int32_t *col, double *val)
{
    int64_t m = (int64_t)nx * ny * nz;
    int64_t acc = 0;
    if (row_ptr) row_ptr[0] = 0;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                acc += (int64_t)span3(x, nx) * span3(y, ny) * span3(z, nz);
                if (row_ptr) row_ptr[((int64_t)z * ny + y) * nx + x + 1] = (int32_t)acc;
            }
    if (!col || !val || !row_ptr) return acc;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int32_t x = (int32_t)(i % nx);
        int32_t y = (int32_t)((i / nx) % ny);
        int32_t z = (int32_t)(i / ((int64_t)nx * ny));
        int64_t k = row_ptr[i];
        for (int dz = -1; dz <= 1; ++dz) {
            if (z + dz < 0 || z + dz >= nz) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                if (y + dy < 0 || y + dy >= ny) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    if (x + dx < 0 || x + dx >= nx) continue;
                    int64_t c = ((int64_t)(z + dz) * ny + (y + dy)) * nx + (x + dx);
                    col[k] = (int32_t)c;
                    val[k] = (c == i) ? 26.0 : -1.0 + 0.01 * sym(seed, ST_VAL, (uint64_t)k);
                    ++k;
                }
            }
        }
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* R-MAT graph (Chakrabarti, Zhan, Faloutsos, SDM 2004): 2^scale rows,  */
/* nedges edges, quadrant probabilities (a, b, c, 1-a-b-c) at each of   */
/* the scale levels, no noise, no permutation.  Duplicate edges merged, */
/* self loops kept.  If inject_len > 0, one seeded row is replaced by   */
/* inject_len distinct uniform sorted columns.  Values U[-1, 1).        */
/* col/val must hold cap entries; returns nnz, or -1 if cap too small   */
/* or memory ran out.  *inject_row receives the injected row (or -1).   */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t synth_rmat(int32_t scale, int64_t nedges, double a, double b, double c,
                   uint64_t seed, int64_t inject_len, int32_t *row_ptr,
                   int32_t *col, double *val, int64_t cap, int32_t *inject_row)
{
    int64_t m = (int64_t)1 << scale;
    int32_t *er = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nedges > 0 ? nedges : 1));
    int32_t *ec = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nedges > 0 ? nedges : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    if (!er || !ec || !cnt || !pos) { free(er); free(ec); free(cnt); free(pos); return -1; }
    const double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        int32_t r = 0, q = 0;
        for (int32_t lv = 0; lv < scale; ++lv) {
            double u = synth_unit(seed, ST_RMAT, (uint64_t)e * (uint64_t)scale + (uint64_t)lv);
            int rb = (u >= ab);                 /* lower half: quadrants c, d */
            int cb = (u >= a && u < ab) || (u >= abc);   /* right half: b, d */
            r = (r << 1) | rb;
            q = (q << 1) | cb;
        }
        er[e] = r;
        ec[e] = q;
    }
    for (int64_t e = 0; e < nedges; ++e) cnt[er[e] + 1]++;
    for (int64_t r = 0; r < m; ++r) cnt[r + 1] += cnt[r];
    memcpy(pos, cnt, sizeof(int64_t) * ((size_t)m + 1));
    int32_t *bucket = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nedges > 0 ? nedges : 1));
    if (!bucket) { free(er); free(ec); free(cnt); free(pos); return -1; }
    for (int64_t e = 0; e < nedges; ++e) bucket[pos[er[e]]++] = ec[e];
    free(er);
    free(ec);
    /* sort + merge duplicates per row; the unique count goes to pos[r] */
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < m; ++r) {
        int32_t *p = bucket + cnt[r];
        int64_t len = cnt[r + 1] - cnt[r];
        if (len > 1) qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t k = 0; k < len; ++k)
            if (u == 0 || p[k] != p[u - 1]) p[u++] = p[k];
        pos[r] = u;
    }
    int64_t inj = -1;
    if (inject_len > 0) {
        if (inject_len > m) inject_len = m;
        inj = (int64_t)below(seed, ST_INJROW, 0, (uint64_t)m);
        pos[inj] = inject_len;
    }
    if (inject_row) *inject_row = (int32_t)inj;
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int64_t r = 0; r < m; ++r) {
        nnz += pos[r];
        if (nnz > 0x7fffffffLL) { free(bucket); free(cnt); free(pos); return -1; }
        row_ptr[r + 1] = (int32_t)nnz;
    }
    if (nnz > cap) { free(bucket); free(cnt); free(pos); return -1; }
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < m; ++r) {
        if (r == inj) continue;
        memcpy(col + row_ptr[r], bucket + cnt[r], sizeof(int32_t) * (size_t)pos[r]);
    }
    if (inj >= 0)
        select_sorted(m, inject_len, seed, ST_INJCOL, 0, col + row_ptr[inj]);
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nnz; ++k)
        val[k] = sym(seed, ST_VAL, (uint64_t)k);
    free(bucket);
    free(cnt);
    free(pos);
    return nnz;
}

/* ------------------------------------------------------------------ */
/* Banded rows: row r holds every column in [max(0, r-k), min(m-1, r+k)] */
/* (half-bandwidth k, 2k+1 entries in interior rows), values U[-1,1).   */
/* col/val may be NULL to count only.  Returns nnz (or -1 past int32).  */
int64_t synth_banded(int32_t m, int32_t k, uint64_t seed, int32_t *row_ptr, int32_t *col,
                     double *val)
{
    int64_t acc = 0;
    row_ptr[0] = 0;
    for (int32_t r = 0; r < m; ++r) {
        int64_t lo = (int64_t)r - k < 0 ? 0 : (int64_t)r - k;
        int64_t hi = (int64_t)r + k > m - 1 ? m - 1 : (int64_t)r + k;
        acc += hi - lo + 1;
        if (acc > 0x7fffffffLL) return -1;
        row_ptr[r + 1] = (int32_t)acc;
    }
    if (!col || !val) return acc;
    #pragma omp parallel for schedule(static)
    for (int32_t r = 0; r < m; ++r) {
        int64_t lo = (int64_t)r - k < 0 ? 0 : (int64_t)r - k;
        int64_t b = row_ptr[r], e = row_ptr[r + 1];
        for (int64_t q = b; q < e; ++q) col[q] = (int32_t)(lo + (q - b));
    }
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < acc; ++q)
        val[q] = sym(seed, ST_VAL, (uint64_t)q);
    return acc;
}

/* Row lengths uniform in {lo..hi} (no forced empty rows); writes         */
/* row_ptr[m+1] and returns nnz (or -1 past int32).  Fill the columns and */
/* values with synth_fill_uniform.                                       */
int64_t synth_range_rows_ptr(int32_t m, int32_t lo, int32_t hi, uint64_t seed, int32_t *row_ptr)
{
    int64_t acc = 0;
    row_ptr[0] = 0;
    for (int32_t r = 0; r < m; ++r) {
        acc += lo + (int64_t)below(seed, ST_LEN, (uint64_t)r, (uint64_t)(hi - lo + 1));
        if (acc > 0x7fffffffLL) return -1;
        row_ptr[r + 1] = (int32_t)acc;
    }
    return acc;
}

/* Block-diagonal with dense blocks: consecutive blocks of size drawn      */
/* uniformly from {bmin..bmax} (the last one cut at m); every entry of a   */
/* block is stored, values U[-1,1).  col/val may be NULL to count only.    */
/* Returns nnz (or -1 past int32).                                        */
int64_t synth_blockdiag(int32_t m, int32_t bmin, int32_t bmax, uint64_t seed,
                        int32_t *row_ptr, int32_t *col, double *val)
{
    int64_t acc = 0;
    int32_t r = 0;
    uint64_t blk = 0;
    row_ptr[0] = 0;
    while (r < m) {
        int32_t b = bmin + (int32_t)below(seed, ST_LEN, blk++, (uint64_t)(bmax - bmin + 1));
        if (b > m - r) b = m - r;
        for (int32_t i = 0; i < b; ++i) {
            acc += b;
            if (acc > 0x7fffffffLL) return -1;
            row_ptr[r + i + 1] = (int32_t)acc;
            if (col) {
                int64_t q = acc - b;
                for (int32_t j = 0; j < b; ++j) col[q + j] = r + j;
            }
        }
        r += b;
    }
    if (val) {
        #pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < acc; ++q)
            val[q] = sym(seed, ST_VAL, (uint64_t)q);
    }
    return acc;
}
