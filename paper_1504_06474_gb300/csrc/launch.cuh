// launch.cuh -- host-side launch of kernels (a), (b), (c) for one precision.
#pragma once
#include <cuda_runtime.h>

#include "layout.h"
#include "segsum.cuh"

namespace ssspmv {

struct Call {
    int32_t m = 0, n = 0, nnz = 0;
    const int32_t *row_ptr = nullptr;
    const int32_t *col = nullptr;
    const void *val = nullptr;
    const void *x = nullptr;
    void *y = nullptr;
    Layout lay;
    unsigned char *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t *ev = nullptr;       // 4 library-owned events or null
    int exact = 0;                   // dirty tiles store in their true rows
    int block_warps = 0;             // warps per block of kernel (b); 0: the most that fit
    int skip_partition = 0;          // plan execution: tile offsets already in the workspace
    double alpha = 1.0, beta = 0.0;  // y = alpha A x + beta y when axpby (exact stores)
    int axpby = 0;
    uint32_t *dbg_desc = nullptr;    // ntiles*W words or null
    void *dbg_yspec = nullptr;       // m values or null
};

int record_cuda_error(cudaError_t e);  // api.cu: remembers e, returns SSSPMV_ECUDA
int device_sm_count();                 // api.cu: SMs of the current device (cached)

constexpr int kZeroBlocks = 32;

// launches a kernel that may start while the kernel before it on the stream
// finishes (programmatic dependent launch): the kernel calls grid_dep_wait()
// before it reads anything that kernel wrote.  Kernels (b) and (c) are
// launched this way, which hides most of a launch's latency.
template <class... Params, class Arg>
cudaError_t launch_dependent(void (*kernel)(Params...), unsigned grid, unsigned block,
                             size_t smem, cudaStream_t stream, const Arg &arg)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, arg);
}

// resident warps per SM of kernel (b) for this tile shape when launched with
// blocks of bw warps (cached per device and block size)
template <class P, int W>
int segsum_resident_warps(int bw)
{
    using SM = WarpSmem<P, W>;
    constexpr BlockShape BS = pick_block_shape(SM::BYTES, P::max_warps(W));
    constexpr int B = BS.B;
    static int cache[64][33] = {{0}};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (bw < 1 || bw > B) bw = B;
    if (cache[dev][bw] > 0) return cache[dev][bw];
    auto kb = segsum_kernel<P, W, B, BS.blocks, false>;
    int nb = 0;
    if (cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, B * SM::BYTES) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kb, bw * 32, bw * SM::BYTES) !=
            cudaSuccess ||
        nb <= 0) {
        (void)cudaGetLastError();
        return bw;  // at least one block
    }
    cache[dev][bw] = nb * bw;
    return cache[dev][bw];
}

// warps per block of kernel (b).  Automatic choice: every warp that fits in
// shared memory for long rows; for short rows (mean below 20 entries, where
// power-law column patterns reuse x heavily) only as many as keep the
// shared-memory carve-out at or below 200 KB and at most the precision's
// kShortRowWarps, so that L1 keeps room for the gathered x.  Measured on
// W = 15: a 27-point stencil runs 3% faster with all 19 FP64 warps (6% with
// 24 FP32 warps); R-MAT scale 22 runs kernel (b) in 359 us with 14 FP64
// warps against 379 with 17 and 576 with 19, and R-MAT scale 20 in FP32
// 8% faster with 16 warps than with 20.
template <class P, int W>
int segsum_block_warps(const Call &c)
{
    using SM = WarpSmem<P, W>;
    constexpr BlockShape BS = pick_block_shape(SM::BYTES, P::max_warps(W));
    constexpr int B = BS.B;
    if (c.block_warps >= 1) return c.block_warps < B ? c.block_warps : B;
    if ((int64_t)c.nnz >= 20 * (int64_t)c.m) return B;
    int l1w = (200 * 1024 - 1024) / SM::BYTES;
    if (l1w > P::kShortRowWarps) l1w = P::kShortRowWarps;
    if (l1w < 1) l1w = 1;
    return l1w < B ? l1w : B;
}

// kernel (c)'s shared memory: one buffer of L+1 partials per warp (the
// repair of a dirty tile), and the attribute that allows it past 48 KB
template <class P>
size_t calib_smem_bytes(int32_t L)
{
    return (size_t)kCalibWarps * (size_t)(L + 1) * sizeof(typename P::y_t);
}

template <class P, bool BATCHED>
cudaError_t calib_smem_attr(size_t smem)
{
    static size_t done[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (done[dev] >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(calibrate_kernel<P, BATCHED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done[dev] = smem;
    return e;
}

// resident blocks of kernel (c) per SM with `smem` bytes of shared memory
// (the occupancy query, once per device and size)
template <class P, bool BATCHED>
int calib_blocks_per_sm(size_t smem)
{
    static int cached[64] = {0};
    static size_t cached_smem[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] > 0 && cached_smem[dev] == smem) return cached[dev];
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, calibrate_kernel<P, BATCHED>,
                                                      kCalibWarps * 32, smem) != cudaSuccess ||
        n < 1) {
        (void)cudaGetLastError();
        n = 1;
    }
    cached_smem[dev] = smem;
    cached[dev] = n;
    return n;
}

// kernel (c)'s grid, one wave so that no block waits for another to finish:
// the synchronizer role (its warps stride over windows of 32 bunches; at
// most a third of the wave), the zeroing role, and the tile role in what is
// left (a warp per tile for small matrices; its warps stride over the dirty
// tiles kernel (b) listed)
template <class P, bool BATCHED>
void calib_grid(CalibArgs &a, int64_t ntiles, int64_t nbunches, int32_t nzero, size_t smem)
{
    const int64_t wave = (int64_t)calib_blocks_per_sm<P, BATCHED>(smem) * device_sm_count();
    int64_t sync = (nbunches + 32 * kCalibWarps - 1) / (32 * kCalibWarps);
    const int64_t sync_cap = wave / 3 > 1 ? wave / 3 : 1;
    if (sync > sync_cap) sync = sync_cap;
    if (sync < 1) sync = 1;
    int64_t tiles = (ntiles + kCalibWarps - 1) / kCalibWarps;
    int64_t room = wave - sync - nzero;
    if (tiles > room) tiles = room;
    if (tiles < 1) tiles = 1;
    a.nblk_sync = (int32_t)sync;
    a.nblk_zero = nzero;
    a.nblk_tiles = (int32_t)tiles;
}

// S (tiles per bunch) and the bunch count for this call
template <class P, int W>
void resolve_bunches(Layout &l, int32_t S_opt)
{
    l.S = S_opt > 0 ? S_opt : auto_bunch_tiles(l.ntiles);
    l.nbunches = (l.ntiles + l.S - 1) / l.S;
}

template <class P, int W>
int run_shape(const Call &c)
{
    using SM = WarpSmem<P, W>;
    constexpr BlockShape BS = pick_block_shape(SM::BYTES, P::max_warps(W));
    constexpr int B = BS.B;
    const Layout &l = c.lay;
    unsigned char *ws = c.ws;
    uint32_t *err = reinterpret_cast<uint32_t *>(ws + l.off_err);
    int32_t *toff = reinterpret_cast<int32_t *>(ws + l.off_tile_offset);
    uint32_t *info = reinterpret_cast<uint32_t *>(ws + l.off_tile_info);
    int32_t *sidx = reinterpret_cast<int32_t *>(ws + l.off_sync_idx);
    void *sval = ws + l.off_sync_val;
    void *tval = ws + l.off_tail_val;
    int32_t *tflag = reinterpret_cast<int32_t *>(ws + l.off_tail_flag);
    cudaError_t e = cudaSuccess;

    if (c.ev && (e = cudaEventRecord(c.ev[0], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    if (c.skip_partition) {
        // the partition is the plan's; the error word, the bunch ticket and
        // the dirty-tile count (cleared by kernel (a) otherwise) start again
        // from zero, the plan's schedule flag stays
        if ((e = cudaMemsetAsync(err, 0, 3 * sizeof(uint32_t), c.stream)) != cudaSuccess)
            return record_cuda_error(e);
    } else {
        launch_partition(c.row_ptr, c.m, c.nnz, l.L, l.ntiles, toff, err, c.stream,
                         partition_method(c.m, l.ntiles));
    }
    if (c.ev && (e = cudaEventRecord(c.ev[1], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    if (l.ntiles > 0) {
        SegsumArgs a;
        a.row_ptr = c.row_ptr;
        a.col = c.col;
        a.val = c.val;
        a.x = c.x;
        a.y = c.y;
        a.tile_offset = toff;
        a.tile_info = info;
        a.sync_idx = sidx;
        a.sync_val = sval;
        a.tail_val = tval;
        a.tail_flag = tflag;
        a.err = err;
        a.ticket = err + kWordTicket;
        a.spread = err + kWordSpread;
        a.dirty_count = err + kWordDirty;
        a.dirty_list = reinterpret_cast<int32_t *>(ws + l.off_dirty_list);
        a.dbg_desc = c.dbg_desc;
        a.m = c.m;
        a.nnz = c.nnz;
        a.ntiles = l.ntiles;
        a.nbunches = l.nbunches;
        a.S = l.S;
        a.alpha = c.alpha;
        a.beta = c.beta;
        a.axpby = c.axpby;
        auto kb = c.exact ? segsum_kernel<P, W, B, BS.blocks, true>
                          : segsum_kernel<P, W, B, BS.blocks, false>;
        static int attr_done[2][64] = {{0}};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !attr_done[c.exact][dev]) {
            e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     B * SM::BYTES);
            if (e != cudaSuccess) return record_cuda_error(e);
            attr_done[c.exact][dev] = 1;
        }
        // one wave of persistent warps; bunches beyond it come from the ticket
        const int bw = segsum_block_warps<P, W>(c);
        int64_t nw = (int64_t)device_sm_count() * segsum_resident_warps<P, W>(bw);
        if (nw > l.nbunches) nw = l.nbunches;
        if (nw < 1) nw = 1;
        const unsigned grid = (unsigned)((nw + bw - 1) / bw);
        e = launch_dependent(kb, grid, bw * 32, bw * SM::BYTES, c.stream, a);
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    if (c.dbg_yspec && c.m > 0) {
        e = cudaMemcpyAsync(c.dbg_yspec, c.y, sizeof(typename P::y_t) * (size_t)c.m,
                            cudaMemcpyDeviceToDevice, c.stream);
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    if (c.ev && (e = cudaEventRecord(c.ev[2], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    {
        CalibArgs a;
        a.row_ptr = c.row_ptr;
        a.tile_offset = toff;
        a.tile_info = info;
        a.sync_idx = sidx;
        a.sync_val = sval;
        a.tail_val = tval;
        a.tail_flag = tflag;
        a.y = c.y;
        a.err = err;
        a.m = c.m;
        a.nnz = c.nnz;
        a.L = l.L;
        a.ntiles = l.ntiles;
        a.nbunches = l.nbunches;
        a.dirty_count = err + kWordDirty;
        a.dirty_list = reinterpret_cast<const int32_t *>(ws + l.off_dirty_list);
        a.alpha = c.alpha;
        a.beta = c.beta;
        a.axpby = c.axpby;
        // the flag of kernel (a) is the plan's when the partition is reused
        a.spread_reset = c.skip_partition ? nullptr : err + kWordSpread;
        const size_t smem = calib_smem_bytes<P>(l.L);
        if ((e = calib_smem_attr<P, false>(smem)) != cudaSuccess) return record_cuda_error(e);
        calib_grid<P, false>(a, l.ntiles, l.nbunches, kZeroBlocks, smem);
        const unsigned grid = (unsigned)(a.nblk_tiles + a.nblk_sync + a.nblk_zero);
        e = launch_dependent(calibrate_kernel<P, false>, grid, kCalibWarps * 32, smem, c.stream, a);
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    if (c.ev && (e = cudaEventRecord(c.ev[3], c.stream)) != cudaSuccess)
        return record_cuda_error(e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_error(e);
    return SSSPMV_OK;
}

}  // namespace ssspmv
