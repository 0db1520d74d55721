// noalloc.cu -- ssspmv_csr_f64_noalloc: the FP64 product with its workspace in
// a fixed device array owned by this library, for callers that cannot
// allocate device memory themselves.
//
// Who needs it: code that is handed device pointers for A, x and y but owns no
// allocator -- a plug-in called from inside another application's solver
// loop, whose device memory belongs to the host application's pool -- and code
// that must not call cudaMalloc/cudaFree on its hot path, because those calls
// can synchronise the whole device and stall every other stream.
//
// Scratch rules: the array below holds the tile offsets, per-tile info and
// synchronizer records of one call (SSSPMV_NOALLOC_SCRATCH_BYTES in total).
// Every GPU that loads this library holds it until the process exits.  All
// calls on a device share it and it keeps the last call's contents.  Each
// call clears the array's 16-byte header on its stream first (the device
// error word, the bunch ticket, the dirty-tile count and kernel (b)'s
// schedule flag, which a call that stopped between kernels (b) and (c) could
// otherwise leave set); the kernels write every other entry before they read
// it.  Calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// the shared array and corrupt each other's results: order them on one
// stream or through events.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress while that device is current and caches it; make that
// first call before any stream capture begins.  `stream` must belong to the
// current device (checked).  cudaDeviceReset unloads the array with the
// module, so the cached address is not valid afterwards: do not call this
// entry point in a process after resetting the device it ran on.  No call
// allocates device memory (no cudaMalloc, cudaFree or allocating library
// routine; the header is cleared with cudaMemsetAsync).
#include <cuda_runtime.h>

#include <mutex>

#include "layout.h"
#include "ssspmv.h"

namespace ssspmv {
int record_cuda_error(cudaError_t e);  // api.cu
int check_csr_args(int32_t m, int32_t n, int32_t nnz, const void *row_ptr, const void *col,
                   const void *val, const void *x, const void *y);  // api.cu
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[SSSPMV_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int ssspmv_csr_f64_noalloc(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                                      const int32_t *col_idx, const double *val, const double *x,
                                      double *y, const ssspmv_opts *opts, void *stream)
{
    // the same verdicts on the arguments and options as ssspmv_csr_f64 (e.g.
    // EUNSUPPORTED for a tile shape that is not compiled in), before anything
    // is queued on the stream
    int rc = ssspmv::check_csr_args(m, n, nnz, row_ptr, col_idx, val, x, y);
    if (rc) return rc;
    rc = ssspmv_plan_shape(m, nnz, 8, opts, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (rc) return rc;
    const size_t need = ssspmv_workspace_bytes(m, nnz, 8, opts);
    if (need == 0) return SSSPMV_EINVAL;
    if (need > (size_t)SSSPMV_NOALLOC_SCRATCH_BYTES) return SSSPMV_ETOOLARGE;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ssspmv::record_cuda_error(e);
    if (dev < 0 || dev >= kMaxDevices) return SSSPMV_EINVAL;
    // the cached address is this device's array: the kernels must run here
    // (the default-stream handles always name the current device)
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
        int sdev = -1;
        e = cudaStreamGetDevice(st, &sdev);
        if (e != cudaSuccess) return ssspmv::record_cuda_error(e);
        if (sdev != dev) return SSSPMV_EINVAL;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            // host code only knows the array by a host-side stand-in; its
            // device address is looked up once, with this device current
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return ssspmv::record_cuda_error(e);
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    if (m > 0) {
        e = cudaMemsetAsync(scratch, 0, ssspmv::kHeaderBytes, st);
        if (e != cudaSuccess) return ssspmv::record_cuda_error(e);
    }
    return ssspmv_csr_f64(m, n, nnz, row_ptr, col_idx, val, x, y, opts, scratch,
                          (size_t)SSSPMV_NOALLOC_SCRATCH_BYTES, stream);
}
