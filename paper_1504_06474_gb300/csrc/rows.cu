// rows.cu -- row-parallel CSR kernels (the CSR-scalar and CSR-vector methods
// the paper describes in Sec. 2.1 and benchmarks against in Sec. 4.3): a
// group of G lanes per row, G = 1 being the scalar kernel (one thread per
// row) and G = 2..32 the vector kernel (the lanes of a group stride over the
// row's entries and combine their sums with shuffles).  They need no partition and no calibration, and beat the
// segmented sum where every row has about the same, small length; they are
// classes the selector can choose.  FP64, FMA accumulation, fixed order:
// runs are deterministic.
#include <cuda_runtime.h>

#include "launch.cuh"

namespace ssspmv {

constexpr int kRowThreads = 256;

template <int G>
__global__ void __launch_bounds__(kRowThreads)
    csr_rows_kernel(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                    const double *__restrict__ val, const double *__restrict__ x,
                    double *__restrict__ y, int32_t m, double alpha, double beta, int32_t axpby)
{
    static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "G is a power of two up to 32");
    constexpr int RPW = 32 / G;  // rows per warp per pass
    const int lane = threadIdx.x & 31;
    const int sub = lane & (G - 1);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the loop bound is the same for every lane of a warp (the shuffles need all)
    for (int64_t r0 = warp * RPW; r0 < m; r0 += nwarps * RPW) {
        const int64_t r = r0 + lane / G;
        double s0 = 0.0, s1 = 0.0;  // two chains: entries sub, sub+2G, ... and sub+G, ...
        if (r < m) {
            const int32_t b = __ldg(row_ptr + r), e = __ldg(row_ptr + r + 1);
            int32_t k = b + sub;
            for (; k + G < e; k += 2 * G) {
                s0 = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s0);
                s1 = fma(__ldg(val + k + G), __ldg(x + __ldg(col + k + G)), s1);
            }
            if (k < e) s0 = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s0);
        }
        double s = s0 + s1;
#pragma unroll
        for (int d = G / 2; d >= 1; d >>= 1) s += __shfl_xor_sync(FULL, s, d);
        if (r < m && sub == 0) y[r] = scaled_store_value(y, r, s, alpha, beta, axpby);
    }
}

// lanes per row for a mean row length: the power of two nearest half the
// mean, so each lane takes about two entries
int rows_group_for(int32_t m, int32_t nnz)
{
    const double mean = m > 0 ? (double)nnz / (double)m : 0.0;
    int g = 1;
    while (g < 32 && 2.0 * g * 1.5 <= mean) g *= 2;
    return g;
}

int run_rows_f64(const Call &c, int group)
{
    cudaError_t e = cudaSuccess;
    if (c.ev && (e = cudaEventRecord(c.ev[0], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    // the workspace's error word starts at zero, as after kernel (a)
    if (c.ws && (e = cudaMemsetAsync(c.ws + c.lay.off_err, 0, 2 * sizeof(uint32_t), c.stream)) !=
                    cudaSuccess)
        return record_cuda_error(e);
    if (c.ev && (e = cudaEventRecord(c.ev[1], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    if (c.m > 0) {
        const int g = group > 0 ? group : rows_group_for(c.m, c.nnz);
        const int64_t threads = (int64_t)c.m * g;
        int64_t blocks = (threads + kRowThreads - 1) / kRowThreads;
        const int64_t cap = 32LL * device_sm_count();
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        const unsigned grid = (unsigned)blocks;
        const double *val = static_cast<const double *>(c.val);
        const double *x = static_cast<const double *>(c.x);
        double *y = static_cast<double *>(c.y);
        switch (g) {
#define X(G)                                                                                   \
    case G:                                                                                    \
        csr_rows_kernel<G><<<grid, kRowThreads, 0, c.stream>>>(c.row_ptr, c.col, val, x, y, c.m, \
                                                               c.alpha, c.beta, c.axpby);      \
        break;
            X(1) X(2) X(4) X(8) X(16) X(32)
#undef X
        default: return SSSPMV_EINVAL;
        }
    }
    if (c.ev && (e = cudaEventRecord(c.ev[2], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    if (c.ev && (e = cudaEventRecord(c.ev[3], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_error(e);
    return SSSPMV_OK;
}

}  // namespace ssspmv
