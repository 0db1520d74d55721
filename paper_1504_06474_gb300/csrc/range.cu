// range.cu -- the product over a contiguous range of tiles, for splitting one
// y = A x across devices.  Shard g owns the nonzeros [B, E) = [b_t0, b_t1) of
// the whole matrix's tiling; it computes every row that lies inside them and
// returns the partial sums of the (at most two) rows cut at its ends.  Adding
// those partials row by row is the synchronization step of Sec. 3.2 and
// Algorithm 1 one level up: between shards instead of between thread-bunches.
//
// The shard runs the ordinary three kernels on a view of the matrix: rows
// [r_first, r_end) with a row-pointer array shifted by B and clamped to
// [0, E - B] (written into the front of the workspace), and col_idx/val
// offset by B.  Its tiles are exactly the whole matrix's tiles [t0, t1)
// (B is a multiple of L), so the index artefacts and the arithmetic of every
// tile are those of the unsplit product.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "layout.h"
#include "ssspmv.h"

namespace ssspmv {

int record_cuda_error(cudaError_t e);  // api.cu
int device_sm_count();                 // api.cu

// tile length of the call (the whole matrix and every shard use the same)
static int range_tile_len(int32_t m, int32_t nnz, const ssspmv_opts *opts, int32_t *L,
                          int64_t *ntiles)
{
    if (opts && opts->variant == SSSPMV_VARIANT_ROWS) return SSSPMV_EUNSUPPORTED;
    int32_t W = 0, Lr = 0, S = 0;
    int64_t nt = 0, nb = 0;
    int rc = ssspmv_plan_shape(m, nnz, 8, opts, &W, &Lr, &S, &nt, &nb);
    if (rc) return rc;
    *L = Lr;
    *ntiles = nt;
    return SSSPMV_OK;
}

__global__ void range_bounds_kernel(const int32_t *__restrict__ row_ptr, int32_t m, int64_t B,
                                    int64_t E, int32_t *out)
{
    // rightmost r in [0, m] with row_ptr[r] <= b, for b = B and b = E
    const int which = threadIdx.x;
    if (which > 1) return;
    const int64_t b = which == 0 ? B : E;
    int32_t lo = 0, hi = m;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if ((int64_t)__ldg(row_ptr + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    out[which] = lo;
}

__global__ void range_shift_kernel(const int32_t *__restrict__ row_ptr, int32_t r_first,
                                   int32_t m_sub, int32_t B, int32_t nnz_sub,
                                   int32_t *__restrict__ sub)
{
    // a valid CSR view whatever bounds the caller gave: it starts at 0, ends
    // at nnz_sub and never decreases (bounds that do not match row_ptr give
    // wrong sums, flagged in the seam record, but no access outside [B, E))
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m_sub; i += stride) {
        int32_t v = __ldg(row_ptr + r_first + i) - B;
        v = v < 0 ? 0 : (v > nnz_sub ? nnz_sub : v);
        if (i == 0) v = 0;
        if (i == m_sub) v = nnz_sub;
        sub[i] = v;
    }
}

// the shard's seam record: its partials of rows r_first and r2 (the row cut
// at E when it is a second cut row, else -1), and whether the bounds given
// match row_ptr (r_first, r_last: the rightmost rows with row_ptr <= B, <= E)
__global__ void range_seam_kernel(const int32_t *__restrict__ row_ptr, int32_t m, int64_t B,
                                  int64_t E, int32_t r_first, int32_t r_last, int32_t r2,
                                  const double *y, ssspmv_seam *seam)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t ok = 1;
    if (__ldg(row_ptr + r_first) > B) ok = 0;
    if (r_first < m && __ldg(row_ptr + r_first + 1) <= B) ok = 0;
    if (__ldg(row_ptr + r_last) > E) ok = 0;
    if (r_last < m && __ldg(row_ptr + r_last + 1) <= E) ok = 0;
    seam->row[0] = r_first < m ? r_first : -1;
    seam->val[0] = r_first < m ? y[r_first] : 0.0;
    seam->row[1] = r2;
    seam->val[1] = r2 >= 0 ? y[r2] : 0.0;
    seam->status = ok ? 0 : SSSPMV_DEV_RANGE;
}

struct RangeView {
    int32_t L = 0;
    int64_t ntiles = 0, B = 0, E = 0;
    int32_t r_end = 0, m_sub = 0, nnz_sub = 0;
    size_t rp_bytes = 0;  // the shifted row pointers at the front of the workspace
};

static int range_view(int32_t m, int32_t nnz, int64_t t0, int64_t t1, int32_t r_first,
                      int32_t r_last, const ssspmv_opts *opts, RangeView &v)
{
    if (m < 0 || nnz < 0) return SSSPMV_EINVAL;
    int rc = range_tile_len(m, nnz, opts, &v.L, &v.ntiles);
    if (rc) return rc;
    if (t0 < 0 || t1 < t0 || t1 > v.ntiles) return SSSPMV_EINVAL;
    v.B = t0 * (int64_t)v.L < nnz ? t0 * (int64_t)v.L : nnz;
    v.E = t1 * (int64_t)v.L < nnz ? t1 * (int64_t)v.L : nnz;
    if (r_first < 0 || r_first > m || r_last < r_first || r_last > m) return SSSPMV_EINVAL;
    v.r_end = r_last < m ? r_last + 1 : m;
    if (v.r_end < r_first) return SSSPMV_EINVAL;
    v.m_sub = v.r_end - r_first;
    v.nnz_sub = (int32_t)(v.E - v.B);
    v.rp_bytes = align256(sizeof(int32_t) * ((size_t)v.m_sub + 1));
    return SSSPMV_OK;
}

}  // namespace ssspmv

using namespace ssspmv;

extern "C" {

int ssspmv_range_bounds(int32_t m, int32_t nnz, const int32_t *row_ptr, const ssspmv_opts *opts,
                        int64_t t0, int64_t t1, int32_t *r_first, int32_t *r_last, void *stream)
{
    if (!row_ptr || !r_first || !r_last || m < 0 || nnz < 0) return SSSPMV_EINVAL;
    int32_t L = 0;
    int64_t ntiles = 0;
    int rc = range_tile_len(m, nnz, opts, &L, &ntiles);
    if (rc) return rc;
    if (t0 < 0 || t1 < t0 || t1 > ntiles) return SSSPMV_EINVAL;
    const int64_t B = t0 * (int64_t)L < nnz ? t0 * (int64_t)L : nnz;
    const int64_t E = t1 * (int64_t)L < nnz ? t1 * (int64_t)L : nnz;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *d = nullptr;
    int32_t h[2] = {0, 0};
    cudaError_t e = cudaMallocAsync(&d, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return record_cuda_error(e);
    range_bounds_kernel<<<1, 32, 0, s>>>(row_ptr, m, B, E, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaError_t f = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = f;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return record_cuda_error(e);
    *r_first = h[0];
    // the row cut at E (the shard's last row) -- the same row as r_first when
    // the shard lies inside one row, and m for the shard that ends the matrix
    *r_last = h[1];
    return SSSPMV_OK;
}

size_t ssspmv_range_workspace_bytes(int32_t m, int32_t nnz, int64_t t0, int64_t t1,
                                    int32_t r_first, int32_t r_last, const ssspmv_opts *opts)
{
    RangeView v;
    if (range_view(m, nnz, t0, t1, r_first, r_last, opts, v)) return 0;
    const size_t ws = ssspmv_workspace_bytes(v.m_sub, v.nnz_sub, 8, opts);
    if (ws == 0) return 0;
    return v.rp_bytes + ws;
}

int ssspmv_csr_f64_range(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                         const int32_t *col_idx, const double *val, const double *x, double *y,
                         int64_t t0, int64_t t1, int32_t r_first, int32_t r_last,
                         ssspmv_seam *seam, const ssspmv_opts *opts, void *workspace,
                         size_t ws_bytes, void *stream)
{
    if (!seam) return SSSPMV_EINVAL;
    if (m < 0 || n < 0 || nnz < 0 || (m == 0 && nnz != 0)) return SSSPMV_EINVAL;
    if (m > 0 && (!row_ptr || !y)) return SSSPMV_EINVAL;
    if (nnz > 0 && (!col_idx || !val || !x || n == 0)) return SSSPMV_EINVAL;
    if (opts && opts->timer) return SSSPMV_EINVAL;
    RangeView v;
    int rc = range_view(m, nnz, t0, t1, r_first, r_last, opts, v);
    if (rc) return rc;
    if (!workspace || ((uintptr_t)workspace & 255u)) return SSSPMV_EWORKSPACE;
    const size_t need = ssspmv_range_workspace_bytes(m, nnz, t0, t1, r_first, r_last, opts);
    if (need == 0 || ws_bytes < need) return SSSPMV_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    unsigned char *w = static_cast<unsigned char *>(workspace);
    int32_t *rp_sub = reinterpret_cast<int32_t *>(w);
    // the shard that starts the matrix also owns the leading empty rows
    if (t0 == 0 && r_first > 0) {
        e = cudaMemsetAsync(y, 0, sizeof(double) * (size_t)r_first, s);
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    if (m > 0) {
        int64_t blocks = ((int64_t)v.m_sub + 1 + 255) / 256;
        const int64_t cap = 4LL * device_sm_count();
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        range_shift_kernel<<<(unsigned)blocks, 256, 0, s>>>(row_ptr, r_first, v.m_sub,
                                                           (int32_t)v.B, v.nnz_sub, rp_sub);
        e = cudaGetLastError();
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    if (v.m_sub > 0) {
        rc = ssspmv_csr_f64(v.m_sub, n, v.nnz_sub, rp_sub, col_idx + v.B, val + v.B, x,
                            y + r_first, opts, w + v.rp_bytes, ws_bytes - v.rp_bytes, stream);
        if (rc) return rc;
    }
    // the cut rows: r_first always (unless the shard is past the last row),
    // r_last when it differs from r_first and is a row of the matrix
    const int32_t r2 = (r_last > r_first && r_last < m) ? r_last : -1;
    range_seam_kernel<<<1, 32, 0, s>>>(row_ptr, m, v.B, v.E, r_first, r_last, r2, y, seam);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_error(e);
    return SSSPMV_OK;
}

int ssspmv_seam_merge(int32_t shards, const ssspmv_seam *seams, int32_t *rows, double *vals,
                      int32_t *count)
{
    if (shards < 0 || (shards > 0 && !seams) || !count) return SSSPMV_EINVAL;
    // partials in shard order; the rows of consecutive records never decrease,
    // so equal rows are adjacent and each row's sum has a fixed order
    int32_t k = 0;
    int32_t last = -1;
    for (int32_t g = 0; g < shards; ++g) {
        if (seams[g].status != 0) return SSSPMV_EDEVICE;
        for (int j = 0; j < 2; ++j) {
            const int32_t r = seams[g].row[j];
            if (r < 0) continue;
            if (r < last) return SSSPMV_EINVAL;
            if (r == last && k > 0) {
                if (vals) vals[k - 1] += seams[g].val[j];
            } else {
                if (rows) rows[k] = r;
                if (vals) vals[k] = seams[g].val[j];
                ++k;
                last = r;
            }
        }
    }
    *count = k;
    return SSSPMV_OK;
}

}  // extern "C"
