// partition.cu -- kernel (a): tile boundaries on row_ptr (Sec. 3.2, Algorithm 1:
// each boundary b_t = min(t*L, nnz) is binary-searched on row_ptr and the
// rightmost match is kept, so a run of empty rows sharing the pointer b_t is
// skipped and the tile starts at the row that holds entry b_t).
#include <cuda_runtime.h>

#include "segsum.cuh"

namespace ssspmv {

constexpr int kPartitionThreads = 256;

__global__ void __launch_bounds__(kPartitionThreads)
    partition_kernel(const int32_t *__restrict__ row_ptr, int32_t m, int32_t nnz, int32_t L,
                     int64_t ntiles, int32_t *__restrict__ tile_offset, uint32_t *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *err = 0u;
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

void launch_partition(const int32_t *row_ptr, int32_t m, int32_t nnz, int32_t L, int64_t ntiles,
                      int32_t *tile_offset, uint32_t *err, cudaStream_t stream)
{
    const int64_t nthreads = ntiles + 1;
    const unsigned grid = (unsigned)((nthreads + kPartitionThreads - 1) / kPartitionThreads);
    partition_kernel<<<grid, kPartitionThreads, 0, stream>>>(row_ptr, m, nnz, L, ntiles,
                                                             tile_offset, err);
}

}  // namespace ssspmv
