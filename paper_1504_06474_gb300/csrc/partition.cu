// partition.cu -- kernel (a): tile boundaries on row_ptr (Sec. 3.2, Algorithm 1:
// each boundary b_t = min(t*L, nnz) is binary-searched on row_ptr and the
// rightmost match is kept, so a run of empty rows sharing the pointer b_t is
// skipped and the tile starts at the row that holds entry b_t).  Two
// launches compute the same array: the per-boundary binary search of the
// paper, and a row-parallel scatter that streams row_ptr once.
#include <cuda_runtime.h>

#include "segsum.cuh"

namespace ssspmv {

int device_sm_count();  // api.cu

constexpr int kPartitionThreads = 256;

__global__ void __launch_bounds__(kPartitionThreads)
    partition_kernel(const int32_t *__restrict__ row_ptr, int32_t m, int32_t nnz, int32_t L,
                     int64_t ntiles, int32_t *__restrict__ tile_offset, uint32_t *err)
{
    grid_dep_trigger();  // kernel (b) may launch its blocks as these finish
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        err[kWordErr] = 0u;
        err[kWordTicket] = 0u;
        err[kWordDirty] = 0u;
        err[kWordSpread] = 1u;  // tiles span 64 rows on average: spread the schedule
    }
    if (t > ntiles) return;
    const int64_t bl = t * (int64_t)L;
    const int32_t b = (int32_t)(bl < nnz ? bl : nnz);
    // invariant: row_ptr[lo] <= b (row_ptr[0] == 0 <= b); answer in [lo, hi]
    int32_t lo = 0, hi = m;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (__ldg(row_ptr + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    tile_offset[t] = lo;
}

// The same partition computed from the rows' side in one streaming pass: the
// boundary b_t < nnz lies in exactly one non-empty row r (row_ptr[r] <= b_t <
// row_ptr[r+1]), which is the rightmost row with row_ptr[r] <= b_t; so each
// non-empty row writes its index to the boundaries it contains.  Reads
// row_ptr once, coalesced, instead of ~log2(m) dependent probes per boundary.
// All index arithmetic is 32-bit (m, nnz and the tile count are below 2^31,
// and r0 + 7 * stride stays below 2^32): the kernel is bound by instruction
// issue, not by its 4 bytes per row.
template <int W>
__global__ void __launch_bounds__(kPartitionThreads)
    partition_scatter_kernel(const int32_t *__restrict__ row_ptr, int32_t m, int32_t nnz,
                             int64_t ntiles, int32_t *__restrict__ tile_offset, uint32_t *err)
{
    constexpr uint32_t L = 32u * W;  // a compile-time divisor
    grid_dep_trigger();  // kernel (b) may launch its blocks as these finish
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t mu = (uint32_t)m;
    if (i0 == 0) {
        err[kWordErr] = 0u;
        err[kWordTicket] = 0u;
        err[kWordDirty] = 0u;
        tile_offset[ntiles] = m;  // b = nnz: every row pointer is <= nnz
    }
    // every lane of a warp runs the same iterations (the ballots need them)
    const uint32_t warp0 = i0 - lane;
    bool spread = false;
    for (uint32_t r0 = i0; warp0 + (r0 - i0) < mu; r0 += 4u * stride) {
        uint32_t lo[4], hi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // four independent rows in flight
            const uint32_t r = r0 + (uint32_t)u * stride;
            const bool in = r < mu;
            lo[u] = in ? (uint32_t)__ldg(row_ptr + r) : 0u;
            hi[u] = in ? (uint32_t)__ldg(row_ptr + r + 1) : 0u;
        }
        // 32 consecutive empty rows (sampled: the first of the four chunks)
        spread = spread || __ballot_sync(0xffffffffu, lo[0] != hi[0] || r0 >= mu) == 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // tiles t with lo <= t*L < hi; a row spanning many tiles is
            // written by the whole warp
            const uint32_t r = r0 + (uint32_t)u * stride;
            const uint32_t tlo = (lo[u] + (L - 1u)) / L;
            const uint32_t thi = (hi[u] + (L - 1u)) / L;
            const bool longrow = thi - tlo > 8u;
            if (!longrow) {
#pragma unroll 1
                for (uint32_t t = tlo; t < thi; ++t) tile_offset[t] = (int32_t)r;
            }
            unsigned lm = __ballot_sync(0xffffffffu, longrow);
            while (lm) {
                const int src = __ffs(lm) - 1;
                lm &= lm - 1;
                const uint32_t a = __shfl_sync(0xffffffffu, tlo, src);
                const uint32_t z = __shfl_sync(0xffffffffu, thi, src);
                const uint32_t rr = __shfl_sync(0xffffffffu, r, src);
                for (uint32_t t = a + lane; t < z; t += 32u) tile_offset[t] = (int32_t)rr;
            }
        }
    }
    // flag for kernel (b)'s schedule (cleared by kernel (c) of the call
    // before), one store per block
    if (__syncthreads_or(spread) && threadIdx.x == 0) err[kWordSpread] = 1u;
}

int partition_method(int32_t m, int64_t ntiles)
{
    // the scatter reads m+1 row pointers once; the search issues ~log2(m)
    // dependent probes per boundary
    return (int64_t)m < 64 * (ntiles + 1) ? 1 : 0;
}

void launch_partition(const int32_t *row_ptr, int32_t m, int32_t nnz, int32_t L, int64_t ntiles,
                      int32_t *tile_offset, uint32_t *err, cudaStream_t stream, int method)
{
    if (method == 1) {
        int64_t blocks = ((int64_t)m + 4 * kPartitionThreads - 1) / (4 * kPartitionThreads);
        const int64_t cap = 32LL * device_sm_count();  // one pass: more rows in flight
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        switch (L / 32) {
#define X(w)                                                                                   \
    case w:                                                                                    \
        partition_scatter_kernel<w><<<(unsigned)blocks, kPartitionThreads, 0, stream>>>(       \
            row_ptr, m, nnz, ntiles, tile_offset, err);                                        \
        return;
            SSSPMV_SHAPES(X)
#undef X
        default: break;  // other tile lengths use the search
        }
    }
    const int64_t nthreads = ntiles + 1;
    const unsigned grid = (unsigned)((nthreads + kPartitionThreads - 1) / kPartitionThreads);
    partition_kernel<<<grid, kPartitionThreads, 0, stream>>>(row_ptr, m, nnz, L, ntiles,
                                                             tile_offset, err);
}

}  // namespace ssspmv
