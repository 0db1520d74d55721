// batched.cu -- many CSR matrices in one pass of the three kernels.
//
// The batch is one global sequence of tiles and bunches: matrix i owns tiles
// [tile_base_i, tile_base_i + ntiles_i) and bunches [bunch_base_i, ...), and
// no bunch crosses a matrix.  Nothing about the batch is known on the host
// beyond an upper bound of its total nonzeros (it sizes the workspace), so a
// set-up kernel reads the caller's device array of descriptors and writes the
// per-matrix records (BatchMat) and the totals; kernel (a) then partitions
// every matrix, the persistent kernel (b) streams every bunch of every matrix
// in one launch, and kernel (c) calibrates them all.  No host synchronisation
// and no allocation: the four launches can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include "launch.cuh"

namespace ssspmv {

constexpr int kPrepThreads = 1024;
constexpr int kBatchPartThreads = 256;

// the descriptor layout of include/ssspmv.h (ssspmv_csr_desc)
struct DescView {
    int32_t m, n, nnz, reserved;
    const int32_t *row_ptr;
    const int32_t *col;
    const void *val;
    const void *x;
    void *y;
};
static_assert(sizeof(DescView) == 56, "ssspmv_csr_desc is 56 bytes");

// exclusive block-wide prefix sum of v over kPrepThreads threads; *total gets the sum
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_sums,
                                                        int64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kPrepThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(FULL, w, d);
            if (lane >= d) w += o;
        }
        warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? warp_sums[warp - 1] : 0) + incl - v;
    *total = warp_sums[kPrepThreads / 32 - 1];
    __syncthreads();
    return before;
}

// One block.  Checks every descriptor (an invalid one is skipped as an empty
// matrix and flagged), numbers the tiles, bunches and rows of the batch, and
// writes the records and totals {tiles, bunches} (totals 0 when the batch
// exceeds the workspace's capacity).  Clears the error word, the ticket and the
// dirty-tile count.
template <int W>
__global__ void __launch_bounds__(kPrepThreads)
    batch_prep_kernel(const DescView *__restrict__ desc, int32_t count, int32_t S,
                      int64_t cap_tiles, int64_t cap_bunches, BatchMat *__restrict__ mats,
                      uint32_t *err, int32_t *totals)
{
    constexpr int32_t L = 32 * W;
    __shared__ int64_t warp_sums[32];
    if (threadIdx.x == 0) {
        err[0] = 0u;
        err[1] = 0u;
        err[kBatchWordDirty] = 0u;
    }
    __syncthreads();
    const int32_t per = (count + kPrepThreads - 1) / kPrepThreads;
    const int32_t i0 = threadIdx.x * per;
    const int32_t i1 = (i0 + per < count) ? i0 + per : count;
    auto valid = [&](const DescView &d) {
        if (d.reserved != 0 || d.m < 0 || d.n < 0 || d.nnz < 0) return false;
        if (d.m > SSSPMV_MAX_DIM || d.nnz > SSSPMV_MAX_DIM) return false;
        if (d.m == 0) return d.nnz == 0;
        if (!d.row_ptr || !d.y) return false;
        if (d.nnz > 0 && (!d.col || !d.val || !d.x || d.n == 0)) return false;
        if (d.nnz > 0 && ((((uintptr_t)d.col) | ((uintptr_t)d.val)) & 15u)) return false;
        return true;
    };
    int64_t nt = 0, nbn = 0, nr = 0;
    bool bad = false;
    for (int32_t i = i0; i < i1; ++i) {
        const DescView d = desc[i];
        if (!valid(d)) {
            bad = true;
            continue;
        }
        const int64_t t = ((int64_t)d.nnz + L - 1) / L;
        nt += t;
        nbn += (t + S - 1) / S;
        nr += d.m;
    }
    if (bad) atomicOr(err, SSSPMV_DEV_BATCH);
    int64_t tot_t = 0, tot_b = 0, tot_r = 0;
    int64_t tb = block_exclusive_scan(nt, warp_sums, &tot_t);
    int64_t bb = block_exclusive_scan(nbn, warp_sums, &tot_b);
    int64_t rb = block_exclusive_scan(nr, warp_sums, &tot_r);
    const bool fits = tot_t <= cap_tiles && tot_b <= cap_bunches;
    for (int32_t i = i0; i < i1; ++i) {
        DescView d = desc[i];
        if (!valid(d)) d = DescView{0, 0, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr};
        const int64_t t = ((int64_t)d.nnz + L - 1) / L;
        BatchMat r;
        r.val = d.val;
        r.col = d.col;
        r.row_ptr = d.row_ptr;
        r.x = d.x;
        r.y = d.y;
        r.m = fits ? d.m : 0;
        r.nnz = fits ? d.nnz : 0;
        r.tile_base = fits ? (int32_t)tb : 0;
        r.bunch_base = fits ? (int32_t)bb : 0;
        r.ntiles = fits ? (int32_t)t : 0;
        r.row_base = (int32_t)(rb < SSSPMV_MAX_DIM ? rb : SSSPMV_MAX_DIM);
        mats[i] = r;
        tb += t;
        bb += (t + S - 1) / S;
        rb += d.m;
    }
    if (threadIdx.x == 0) {
        totals[0] = fits ? (int32_t)tot_t : 0;
        totals[1] = fits ? (int32_t)tot_b : 0;
        if (!fits) atomicOr(err, SSSPMV_DEV_BATCH);
    }
}

// Kernel (a) for a batch: every tile boundary of every matrix (matrix i's
// ntiles_i + 1 offsets start at global position tile_base_i + i), each by the
// rightmost-match binary search on that matrix's row_ptr (Sec. 3.2), and the
// matrix of every global bunch.
template <int W>
__global__ void __launch_bounds__(kBatchPartThreads)
    batch_partition_kernel(const BatchMat *__restrict__ mats, int32_t count,
                           const int32_t *__restrict__ totals, int32_t *__restrict__ tile_offset,
                           int32_t *__restrict__ bunch_mat)
{
    constexpr int32_t L = 32 * W;
    const int64_t nbound = (int64_t)__ldg(totals) + count;
    const int64_t nbun = __ldg(totals + 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nbound; j += stride) {
        int32_t lo = 0, hi = count - 1;  // last matrix whose first offset is at or before j
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo + 1) >> 1);
            if ((int64_t)__ldg(&mats[mid].tile_base) + mid <= j) lo = mid;
            else hi = mid - 1;
        }
        const BatchMat *mm = mats + lo;
        const int64_t k = j - ((int64_t)__ldg(&mm->tile_base) + lo);
        const int32_t nnz = __ldg(&mm->nnz), m = __ldg(&mm->m);
        const int32_t b = (int32_t)(k * L < nnz ? k * L : nnz);
        const int32_t *rp = ldg_ptr(&mm->row_ptr);
        int32_t a = 0, z = m;  // row_ptr[a] <= b (row_ptr[0] == 0)
        while (a < z) {
            const int32_t mid = a + ((z - a + 1) >> 1);
            if (__ldg(rp + mid) <= b) a = mid;
            else z = mid - 1;
        }
        tile_offset[j] = a;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nbun; j += stride) {
        int32_t lo = 0, hi = count - 1;
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo + 1) >> 1);
            if ((int64_t)__ldg(&mats[mid].bunch_base) <= j) lo = mid;
            else hi = mid - 1;
        }
        bunch_mat[j] = lo;
    }
}

template <class P, int W>
int run_batched_shape(int32_t count, const void *desc, const BatchLayout &l, unsigned char *ws,
                      cudaStream_t stream, int exact, int block_warps, cudaEvent_t *ev)
{
    using SM = WarpSmem<P, W>;
    constexpr BlockShape BS = pick_block_shape(SM::BYTES, P::kBatchMaxWarps);
    constexpr int B = BS.B;
    uint32_t *err = reinterpret_cast<uint32_t *>(ws + l.off_err);
    int32_t *totals = reinterpret_cast<int32_t *>(ws + l.off_err + 8);
    BatchMat *mats = reinterpret_cast<BatchMat *>(ws + l.off_mats);
    int32_t *toff = reinterpret_cast<int32_t *>(ws + l.off_toff);
    uint32_t *info = reinterpret_cast<uint32_t *>(ws + l.off_info);
    int32_t *bmat = reinterpret_cast<int32_t *>(ws + l.off_bmat);
    int32_t *sidx = reinterpret_cast<int32_t *>(ws + l.off_sidx);
    cudaError_t e = cudaSuccess;
    const int sms = device_sm_count();

    if (ev && (e = cudaEventRecord(ev[0], stream)) != cudaSuccess) return record_cuda_error(e);
    batch_prep_kernel<W><<<1, kPrepThreads, 0, stream>>>(
        static_cast<const DescView *>(desc), count, l.S, l.cap_tiles, l.cap_bunches, mats, err,
        totals);
    {
        int64_t blocks = (l.cap_tiles + count + kBatchPartThreads - 1) / kBatchPartThreads;
        if (blocks > 8LL * sms) blocks = 8LL * sms;
        if (blocks < 1) blocks = 1;
        batch_partition_kernel<W><<<(unsigned)blocks, kBatchPartThreads, 0, stream>>>(
            mats, count, totals, toff, bmat);
    }
    if (ev && (e = cudaEventRecord(ev[1], stream)) != cudaSuccess) return record_cuda_error(e);
    {
        SegsumArgs a;
        a.row_ptr = nullptr;
        a.col = nullptr;
        a.val = nullptr;
        a.x = nullptr;
        a.y = nullptr;
        a.tile_offset = toff;
        a.tile_info = info;
        a.sync_idx = sidx;
        a.sync_val = ws + l.off_sval;
        a.tail_val = ws + l.off_tval;
        a.tail_flag = reinterpret_cast<int32_t *>(ws + l.off_tflag);
        a.err = err;
        a.ticket = err + 1;
        a.dirty_count = err + kBatchWordDirty;
        a.dirty_list = reinterpret_cast<int32_t *>(ws + l.off_dirty);
        a.dbg_desc = nullptr;
        a.m = 0;
        a.nnz = 0;
        a.ntiles = 0;  // the kernel reads the totals
        a.nbunches = 0;
        a.S = l.S;
        a.mats = mats;
        a.bunch_mat = bmat;
        a.totals = totals;
        auto kb = exact ? segsum_kernel<P, W, B, BS.blocks, true, true>
                        : segsum_kernel<P, W, B, BS.blocks, false, true>;
        static int attr_done[2][64] = {{0}};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !attr_done[exact][dev]) {
            e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     B * SM::BYTES);
            if (e != cudaSuccess) return record_cuda_error(e);
            attr_done[exact][dev] = 1;
        }
        const int bw = (block_warps >= 1 && block_warps <= B) ? block_warps : B;
        int64_t nw = (int64_t)sms * segsum_resident_warps<P, W>(bw);
        if (nw > l.cap_bunches) nw = l.cap_bunches;
        if (nw < 1) nw = 1;
        const unsigned grid = (unsigned)((nw + bw - 1) / bw);
        kb<<<grid, bw * 32, bw * SM::BYTES, stream>>>(a);
    }
    if (ev && (e = cudaEventRecord(ev[2], stream)) != cudaSuccess) return record_cuda_error(e);
    {
        CalibArgs a;
        a.row_ptr = nullptr;
        a.tile_offset = toff;
        a.tile_info = info;
        a.sync_idx = sidx;
        a.sync_val = ws + l.off_sval;
        a.tail_val = ws + l.off_tval;
        a.tail_flag = reinterpret_cast<int32_t *>(ws + l.off_tflag);
        a.y = nullptr;
        a.err = err;
        a.m = 0;
        a.nnz = 0;
        a.L = l.L;
        a.ntiles = 0;
        a.nbunches = 0;
        a.mats = mats;
        a.bunch_mat = bmat;
        a.totals = totals;
        a.count = count;
        a.dirty_count = err + kBatchWordDirty;
        a.dirty_list = reinterpret_cast<const int32_t *>(ws + l.off_dirty);
        const size_t smem = calib_smem_bytes<P>(l.L);
        if ((e = calib_smem_attr<P, true>(smem)) != cudaSuccess) return record_cuda_error(e);
        // a warp per matrix zeroes its leading empty rows
        int32_t nzero = (count + kCalibWarps - 1) / kCalibWarps;
        if (nzero > kZeroBlocks) nzero = kZeroBlocks;
        if (nzero < 1) nzero = 1;
        calib_grid<P, true>(a, l.cap_tiles, l.cap_bunches, nzero, smem);
        const unsigned grid = (unsigned)(a.nblk_tiles + a.nblk_sync + a.nblk_zero);
        calibrate_kernel<P, true><<<grid, kCalibWarps * 32, smem, stream>>>(a);
    }
    if (ev && (e = cudaEventRecord(ev[3], stream)) != cudaSuccess) return record_cuda_error(e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_error(e);
    return SSSPMV_OK;
}

int f32_run_batched(int32_t count, const void *desc, const BatchLayout &l, unsigned char *ws,
                    cudaStream_t stream, int exact, int block_warps, cudaEvent_t *ev)
{
    switch (l.W) {
#define X(w)                                                                                   \
    case w: return run_batched_shape<F32C, w>(count, desc, l, ws, stream, exact, block_warps, ev);
        SSSPMV_SHAPES(X)
#undef X
    default: return SSSPMV_EUNSUPPORTED;
    }
}

}  // namespace ssspmv
