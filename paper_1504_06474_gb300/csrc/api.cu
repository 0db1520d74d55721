// api.cu -- the extern "C" boundary declared in include/ssspmv.h: argument
// checks, tile-shape resolution, workspace carve-up and dispatch to the
// per-precision launchers.  No exception crosses the boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>
#include <mutex>
#include <cstdint>
#include <cstring>
#include <new>

#include "launch.cuh"

namespace ssspmv {

int f64_supported_w(int32_t *out, int cap);
int f64_resolve(Layout &l, int32_t S_opt);
int f64_run(Call &c);
int f32_supported_w(int32_t *out, int cap);
int f32_resolve(Layout &l, int32_t S_opt);
int f32_run(Call &c);
int bf16_supported_w(int32_t *out, int cap);
int bf16_resolve(Layout &l, int32_t S_opt);
int bf16_run(Call &c);
int run_rows_f64(const Call &c, int group);  // rows.cu
int f32_run_batched(int32_t count, const void *desc, const BatchLayout &l, unsigned char *ws,
                    cudaStream_t stream, int exact, int block_warps, cudaEvent_t *ev);  // batched.cu

// one entry per stored value type; the value size identifies the precision
struct Prec {
    int32_t val_bytes;
    int (*supported)(int32_t *, int);
    int (*resolve)(Layout &, int32_t);
    int (*run)(Call &);
};
static const Prec kPrecs[] = {
    {8, f64_supported_w, f64_resolve, f64_run},
    {4, f32_supported_w, f32_resolve, f32_run},
    {2, bf16_supported_w, bf16_resolve, bf16_run},
};

static const Prec *prec_for(int32_t val_bytes)
{
    for (const Prec &p : kPrecs)
        if (p.val_bytes == val_bytes) return &p;
    return nullptr;
}

static thread_local int g_last_cuda_error = 0;

int record_cuda_error(cudaError_t e)
{
    g_last_cuda_error = (int)e;
    return SSSPMV_ECUDA;
}

int device_sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return 152;
    }
    if (cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        (void)cudaGetLastError();
        return 152;
    }
    cache[dev] = n;
    return n;
}

// W from the options, or from the mean row length (odd, snapped to the
// nearest compiled shape): lanes then tend to start at row heads, which keeps
// the x gathers of one warp instruction on neighbouring rows.
static int resolve_w(int32_t m, int32_t nnz, int32_t val_bytes, const ssspmv_opts *o, int32_t *W)
{
    int32_t ws[16];
    const Prec *pr = prec_for(val_bytes);
    if (!pr) return SSSPMV_EUNSUPPORTED;
    int n = pr->supported(ws, 16);
    if (n <= 0) return SSSPMV_EUNSUPPORTED;
    if (n > 16) n = 16;
    if (o && o->W != 0) {
        for (int i = 0; i < n; ++i)
            if (ws[i] == o->W) { *W = o->W; return SSSPMV_OK; }
        return o->W < 0 ? SSSPMV_EINVAL : SSSPMV_EUNSUPPORTED;
    }
    // default: the shortest compiled tile.  Shorter tiles leave room for more
    // resident warps per SM, which hides the latency of the per-tile work
    // (descriptor, gathers, cross-lane sums) better than longer tiles
    // amortise it; this held on stencil and power-law matrices alike, in
    // every precision but one: BF16 values fit as many warps per SM at W = 27
    // as at 15, and with rows of 20 entries or more on average the longer
    // tile is faster (27-point stencil 160^3: 8%; power-law rows: slower)
    int best = ws[0];
    for (int i = 1; i < n; ++i)
        if (ws[i] < best) best = ws[i];
    if (val_bytes == 2 && m > 0 && (int64_t)nnz >= 20 * (int64_t)m)
        for (int i = 0; i < n; ++i)
            if (ws[i] == 27) best = 27;
    *W = best;
    return SSSPMV_OK;
}

// device-independent part of the layout: tile shape, tile count, bunch cap
static int make_layout(int32_t m, int32_t nnz, int32_t val_bytes, const ssspmv_opts *o, Layout &l)
{
    if (m < 0 || nnz < 0) return SSSPMV_EINVAL;
    // the kernels index rows and entries in 32 bits with up to 256 of headroom
    if (m > SSSPMV_MAX_DIM || nnz > SSSPMV_MAX_DIM) return SSSPMV_EINVAL;
    if (o && (o->S < 0 || o->block_warps < 0 || o->variant < 0 || o->variant > 3))
        return SSSPMV_EINVAL;
    if (o && o->variant == SSSPMV_VARIANT_ROWS) {
        // row-parallel kernels: W is the lanes per row; the workspace holds
        // only the error word
        if (val_bytes != 8) return SSSPMV_EUNSUPPORTED;
        if (o->W < 0 || o->W > 32 || (o->W & (o->W - 1))) return SSSPMV_EINVAL;
        l.W = o->W;
        l.L = 0;
        l.ntiles = 0;
        l.nbunch_cap = 0;
        carve(l);
        return SSSPMV_OK;
    }
    int32_t W = 0;
    int rc = resolve_w(m, nnz, val_bytes, o, &W);
    if (rc) return rc;
    l.W = W;
    l.L = 32 * W;
    l.ntiles = ((int64_t)nnz + l.L - 1) / l.L;
    const int32_t S = (o && o->S > 0) ? o->S : auto_bunch_tiles(l.ntiles);
    l.nbunch_cap = (l.ntiles + S - 1) / S;
    carve(l);
    return SSSPMV_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace ssspmv

struct ssspmv_timer {
    int32_t capacity = 0;
    int32_t used = 0;
    cudaEvent_t *ev = nullptr;  // 4 per slot
};

namespace ssspmv {

// the 4 events of the timer's next slot, or null when it is full
static cudaEvent_t *timer_next_slot(ssspmv_timer *t)
{
    if (!t || t->used >= t->capacity) return nullptr;
    return t->ev + 4 * (t->used++);
}

int check_csr_args(int32_t m, int32_t n, int32_t nnz, const void *row_ptr, const void *col,
                   const void *val, const void *x, const void *y)
{
    if (m < 0 || n < 0 || nnz < 0) return SSSPMV_EINVAL;
    if (m == 0 && nnz != 0) return SSSPMV_EINVAL;
    if (m > 0 && (!row_ptr || !y)) return SSSPMV_EINVAL;
    if (nnz > 0 && (!col || !val || !x || n == 0)) return SSSPMV_EINVAL;
    if (nnz > 0 && (!aligned16(col) || !aligned16(val))) return SSSPMV_EINVAL;
    return SSSPMV_OK;
}

// ---------------------------------------------------------------------------
// library-owned workspaces, one per (device, stream), grown stream-ordered

namespace {
struct CachedWs {
    int dev;
    void *stream;
    void *base;    // what cudaMallocAsync returned
    void *ptr;     // 256-byte aligned start
    size_t bytes;  // usable bytes from ptr
};
std::mutex g_ws_mutex;
std::vector<CachedWs> g_ws;
}  // namespace

static int cached_workspace(size_t need, void *stream, void **ptr, size_t *bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda_error(e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    CachedWs *slot = nullptr;
    for (auto &w : g_ws)
        if (w.dev == dev && w.stream == stream) slot = &w;
    if (slot && slot->bytes >= need) {
        *ptr = slot->ptr;
        *bytes = slot->bytes;
        return SSSPMV_OK;
    }
    if (slot && slot->base) {
        // calls already queued on this stream finish with the old buffer first
        if ((e = cudaFreeAsync(slot->base, s)) != cudaSuccess) return record_cuda_error(e);
        slot->base = slot->ptr = nullptr;
        slot->bytes = 0;
    }
    const size_t want = need + need / 4 + 256;  // room to grow a little
    void *base = nullptr;
    if ((e = cudaMallocAsync(&base, want, s)) != cudaSuccess) return record_cuda_error(e);
    if (!slot) {
        g_ws.push_back(CachedWs{dev, stream, nullptr, nullptr, 0});
        slot = &g_ws.back();
    }
    const uintptr_t a = ((uintptr_t)base + 255u) & ~(uintptr_t)255u;
    slot->base = base;
    slot->ptr = reinterpret_cast<void *>(a);
    slot->bytes = want - (a - (uintptr_t)base);
    // the error words at the front start cleared (kernel (b)'s schedule
    // flag is read before the first call's kernel (c) clears it)
    if ((e = cudaMemsetAsync(slot->ptr, 0, kHeaderBytes, s)) != cudaSuccess) return record_cuda_error(e);
    *ptr = slot->ptr;
    *bytes = slot->bytes;
    return SSSPMV_OK;
}

static int run_call(int32_t val_bytes, int32_t m, int32_t n, int32_t nnz,
                    const int32_t *row_ptr, const int32_t *col, const void *val, const void *x,
                    void *y, const ssspmv_opts *opts, void *ws, size_t ws_bytes, void *stream,
                    uint32_t *dbg_desc, void *dbg_yspec, Layout *out_layout,
                    double alpha = 1.0, double beta = 0.0, int axpby = 0)
{
    const Prec *pr = prec_for(val_bytes);
    if (!pr) return SSSPMV_EUNSUPPORTED;
    int rc = check_csr_args(m, n, nnz, row_ptr, col, val, x, y);
    if (rc) return rc;
    Layout l;
    rc = make_layout(m, nnz, val_bytes, opts, l);
    if (rc) return rc;
    if (out_layout) *out_layout = l;
    if (m == 0) return SSSPMV_OK;
    if (!ws) {
        rc = cached_workspace(l.total, stream, &ws, &ws_bytes);
        if (rc) return rc;
    }
    if (ws_bytes < l.total || ((uintptr_t)ws & 255u)) return SSSPMV_EWORKSPACE;
    if (opts && opts->variant == SSSPMV_VARIANT_ROWS) {
        if (dbg_desc || dbg_yspec) return SSSPMV_EINVAL;  // no tiles to export
        Call c;
        c.m = m;
        c.n = n;
        c.nnz = nnz;
        c.row_ptr = row_ptr;
        c.col = col;
        c.val = val;
        c.x = x;
        c.y = y;
        c.lay = l;
        c.ws = static_cast<unsigned char *>(ws);
        c.stream = static_cast<cudaStream_t>(stream);
        c.ev = opts->timer ? timer_next_slot(static_cast<ssspmv_timer *>(opts->timer)) : nullptr;
        c.alpha = alpha;
        c.beta = beta;
        c.axpby = axpby;
        return run_rows_f64(c, l.W);
    }
    rc = pr->resolve(l, opts ? opts->S : 0);
    if (rc) return rc;
    if (l.nbunches > l.nbunch_cap) return SSSPMV_EWORKSPACE;
    if (out_layout) *out_layout = l;
    Call c;
    c.m = m;
    c.n = n;
    c.nnz = nnz;
    c.row_ptr = row_ptr;
    c.col = col;
    c.val = val;
    c.x = x;
    c.y = y;
    c.lay = l;
    c.ws = static_cast<unsigned char *>(ws);
    c.stream = static_cast<cudaStream_t>(stream);
    c.ev = (opts && opts->timer) ? timer_next_slot(static_cast<ssspmv_timer *>(opts->timer))
                                 : nullptr;
    c.dbg_desc = dbg_desc;
    c.dbg_yspec = dbg_yspec;
    c.exact = (opts && opts->variant == SSSPMV_VARIANT_EXACT) ? 1 : 0;
    c.block_warps = opts ? opts->block_warps : 0;
    if (axpby) {
        // speculative stores would overwrite y before its old values are
        // read: scaled products always store exactly
        c.exact = 1;
        c.alpha = alpha;
        c.beta = beta;
        c.axpby = 1;
    }
    return pr->run(c);
}

// ---------------------------------------------------------------------------
// CSR structure check (used by ssspmv_validate_csr)

__global__ void validate_kernel(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                                const int32_t *col, uint32_t *bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0 && (row_ptr[0] != 0 || row_ptr[m] != nnz)) atomicOr(bad, 1u);
    for (int64_t r = i0; r < m; r += stride)
        if (row_ptr[r + 1] < row_ptr[r]) atomicOr(bad, 2u);
    for (int64_t k = i0; k < nnz; k += stride) {
        const int32_t c = col[k];
        if (c < 0 || c >= n) atomicOr(bad, 4u);
    }
}

}  // namespace ssspmv

using namespace ssspmv;

extern "C" {

int ssspmv_version(void) { return 10000; }

int ssspmv_timer_create(int32_t capacity, ssspmv_timer **out)
{
    if (!out || capacity <= 0) return SSSPMV_EINVAL;
    *out = nullptr;
    ssspmv_timer *t = new (std::nothrow) ssspmv_timer;
    if (!t) return SSSPMV_EINVAL;
    t->ev = new (std::nothrow) cudaEvent_t[4 * (size_t)capacity];
    if (!t->ev) { delete t; return SSSPMV_EINVAL; }
    for (int32_t i = 0; i < 4 * capacity; ++i) {
        cudaError_t e = cudaEventCreate(&t->ev[i]);
        if (e != cudaSuccess) {
            for (int32_t j = 0; j < i; ++j) cudaEventDestroy(t->ev[j]);
            delete[] t->ev;
            delete t;
            return record_cuda_error(e);
        }
    }
    t->capacity = capacity;
    *out = t;
    return SSSPMV_OK;
}

void ssspmv_timer_destroy(ssspmv_timer *t)
{
    if (!t) return;
    for (int32_t i = 0; i < 4 * t->capacity; ++i) cudaEventDestroy(t->ev[i]);
    delete[] t->ev;
    delete t;
}

void ssspmv_timer_reset(ssspmv_timer *t)
{
    if (t) t->used = 0;
}

int ssspmv_timer_read(ssspmv_timer *t, float *ms, int32_t cap, int32_t *count)
{
    if (!t) return SSSPMV_EINVAL;
    const int32_t n = t->used < cap ? t->used : cap;
    if (count) *count = t->used;
    for (int32_t i = 0; i < n; ++i) {
        cudaEvent_t *e = t->ev + 4 * i;
        cudaError_t r = cudaEventSynchronize(e[3]);
        float a = 0, b = 0, c = 0, w = 0;
        if (r == cudaSuccess) r = cudaEventElapsedTime(&a, e[0], e[1]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&b, e[1], e[2]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&c, e[2], e[3]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&w, e[0], e[3]);
        if (r != cudaSuccess) return record_cuda_error(r);
        if (ms) {
            ms[4 * i + 0] = a;
            ms[4 * i + 1] = b;
            ms[4 * i + 2] = c;
            ms[4 * i + 3] = w;
        }
    }
    return SSSPMV_OK;
}

int ssspmv_last_cuda_error(void) { return g_last_cuda_error; }

const char *ssspmv_strerror(int code)
{
    switch (code) {
    case SSSPMV_OK: return "success";
    case SSSPMV_EINVAL: return "invalid argument";
    case SSSPMV_EWORKSPACE: return "workspace missing, misaligned or too small";
    case SSSPMV_ECUDA: return "CUDA error (see ssspmv_last_cuda_error)";
    case SSSPMV_EDEVICE: return "a kernel reported an error";
    case SSSPMV_EUNSUPPORTED: return "tile shape not compiled into the library";
    case SSSPMV_ETOOLARGE:
        return "problem exceeds the fixed scratch of ssspmv_csr_f64_noalloc "
               "(SSSPMV_NOALLOC_SCRATCH_BYTES)";
    default: return "unknown error";
    }
}

int ssspmv_supported_w(int32_t *out, int32_t cap, int32_t *count)
{
    int32_t tmp[16];
    int n = f64_supported_w(tmp, 16);
    if (count) *count = n;
    if (out)
        for (int i = 0; i < n && i < cap; ++i) out[i] = tmp[i];
    return SSSPMV_OK;
}

int ssspmv_plan_shape(int32_t m, int32_t nnz, int32_t val_bytes, const ssspmv_opts *opts,
                      int32_t *W, int32_t *L, int32_t *S, int64_t *ntiles, int64_t *nbunches)
{
    const Prec *pr = prec_for(val_bytes);
    if (!pr) return SSSPMV_EUNSUPPORTED;
    Layout l;
    int rc = make_layout(m, nnz, val_bytes, opts, l);
    if (rc) return rc;
    if (opts && opts->variant == SSSPMV_VARIANT_ROWS) {
        if (W) *W = l.W;  // lanes per row (0: chosen per call from nnz/m)
        if (L) *L = 0;
        if (S) *S = 0;
        if (ntiles) *ntiles = 0;
        if (nbunches) *nbunches = 0;
        return SSSPMV_OK;
    }
    rc = pr->resolve(l, opts ? opts->S : 0);
    if (rc) return rc;
    if (W) *W = l.W;
    if (L) *L = l.L;
    if (S) *S = l.S;
    if (ntiles) *ntiles = l.ntiles;
    if (nbunches) *nbunches = l.nbunches;
    return SSSPMV_OK;
}

size_t ssspmv_workspace_bytes(int32_t m, int32_t nnz, int32_t val_bytes, const ssspmv_opts *opts)
{
    if (!prec_for(val_bytes)) return 0;
    Layout l;
    if (make_layout(m, nnz, val_bytes, opts, l)) return 0;
    return l.total;
}

int ssspmv_csr_f64(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                   const int32_t *col_idx, const double *val, const double *x, double *y,
                   const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream)
{
    return run_call(8, m, n, nnz, row_ptr, col_idx, val, x, y, opts, workspace, ws_bytes, stream,
                    nullptr, nullptr, nullptr);
}

int ssspmv_csr_f32(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                   const int32_t *col_idx, const float *val, const float *x, float *y,
                   const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream)
{
    return run_call(4, m, n, nnz, row_ptr, col_idx, val, x, y, opts, workspace, ws_bytes, stream,
                    nullptr, nullptr, nullptr);
}

int ssspmv_csr_bf16f32(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                       const int32_t *col_idx, const uint16_t *val, const float *x, float *y,
                       const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream)
{
    return run_call(2, m, n, nnz, row_ptr, col_idx, val, x, y, opts, workspace, ws_bytes, stream,
                    nullptr, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// batches

static int make_batch_layout(int32_t count, int64_t total_nnz, int32_t val_bytes,
                             const ssspmv_opts *o, BatchLayout &l)
{
    if (count < 0 || total_nnz < 0) return SSSPMV_EINVAL;
    if (o && o->variant == SSSPMV_VARIANT_ROWS) return SSSPMV_EUNSUPPORTED;
    if (o && (o->S < 0 || o->block_warps < 0 || o->variant < 0 || o->variant > 2))
        return SSSPMV_EINVAL;
    int32_t W = 0;
    int rc = resolve_w(0, 0, val_bytes, o, &W);
    if (rc) return rc;
    const int32_t S = (o && o->S > 0) ? o->S : kDefaultS;
    // global tile and bunch numbers are 32-bit in the kernels
    if (total_nnz / (32 * W) + count > (int64_t)SSSPMV_MAX_DIM) return SSSPMV_EINVAL;
    batch_layout(count, total_nnz, W, S, l);
    return SSSPMV_OK;
}

size_t ssspmv_batched_workspace_bytes(int32_t count, int64_t total_nnz, int32_t val_bytes,
                                      const ssspmv_opts *opts)
{
    if (val_bytes != 4) return 0;
    BatchLayout l;
    if (make_batch_layout(count, total_nnz, val_bytes, opts, l)) return 0;
    return l.total;
}

int ssspmv_csr_batched_f32(int32_t count, const ssspmv_csr_desc *mats, int64_t total_nnz,
                           const ssspmv_opts *opts, void *workspace, size_t ws_bytes,
                           void *stream)
{
    BatchLayout l;
    int rc = make_batch_layout(count, total_nnz, 4, opts, l);
    if (rc) return rc;
    if (count == 0) return SSSPMV_OK;
    if (!mats || ((uintptr_t)mats & 7u)) return SSSPMV_EINVAL;
    if (!workspace || ws_bytes < l.total || ((uintptr_t)workspace & 255u))
        return SSSPMV_EWORKSPACE;
    cudaEvent_t *ev = (opts && opts->timer)
                          ? timer_next_slot(static_cast<ssspmv_timer *>(opts->timer))
                          : nullptr;
    return f32_run_batched(count, mats, l, static_cast<unsigned char *>(workspace),
                           static_cast<cudaStream_t>(stream),
                           (opts && opts->variant == SSSPMV_VARIANT_EXACT) ? 1 : 0,
                           opts ? opts->block_warps : 0, ev);
}

// ---------------------------------------------------------------------------
// plans: kernel (a) once, kernels (b) and (c) per execution

struct ssspmv_plan {
    int32_t m = 0, n = 0, nnz = 0, val_bytes = 0;
    const int32_t *row_ptr = nullptr;
    Layout lay;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool owns_ws = false;
    int exact = 0, block_warps = 0, dev = 0;
};

int ssspmv_plan_create(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                       int32_t val_bytes, const ssspmv_opts *opts, void *workspace,
                       size_t ws_bytes, void *stream, ssspmv_plan **out)
{
    if (!out) return SSSPMV_EINVAL;
    *out = nullptr;
    const Prec *pr = prec_for(val_bytes);
    if (!pr) return SSSPMV_EUNSUPPORTED;
    if (m < 0 || n < 0 || nnz < 0 || (m == 0 && nnz != 0)) return SSSPMV_EINVAL;
    if (m > 0 && !row_ptr) return SSSPMV_EINVAL;
    if (opts && opts->timer) return SSSPMV_EINVAL;  // time executions, not the plan
    if (opts && opts->variant == SSSPMV_VARIANT_ROWS) return SSSPMV_EUNSUPPORTED;
    Layout l;
    int rc = make_layout(m, nnz, val_bytes, opts, l);
    if (rc) return rc;
    rc = pr->resolve(l, opts ? opts->S : 0);
    if (rc) return rc;
    ssspmv_plan *p = new (std::nothrow) ssspmv_plan;
    if (!p) return SSSPMV_EINVAL;
    p->m = m;
    p->n = n;
    p->nnz = nnz;
    p->val_bytes = val_bytes;
    p->row_ptr = row_ptr;
    p->lay = l;
    p->exact = (opts && opts->variant == SSSPMV_VARIANT_EXACT) ? 1 : 0;
    p->block_warps = opts ? opts->block_warps : 0;
    if (workspace && (ws_bytes < l.total || ((uintptr_t)workspace & 255u))) {
        delete p;
        return SSSPMV_EWORKSPACE;
    }
    cudaError_t e = cudaGetDevice(&p->dev);
    if (e != cudaSuccess) {
        delete p;
        return record_cuda_error(e);
    }
    if (workspace) {
        p->ws = workspace;
        p->ws_bytes = ws_bytes;
    } else if (l.total > 0) {
        e = cudaMalloc(&p->ws, l.total);
        if (e != cudaSuccess) {
            delete p;
            return record_cuda_error(e);
        }
        p->ws_bytes = l.total;
        p->owns_ws = true;
    }
    if (m > 0) {
        // kernel (a) alone: the tile offsets (and a cleared error word/ticket;
        // the schedule flag it may set starts cleared)
        unsigned char *w = static_cast<unsigned char *>(p->ws);
        e = cudaMemsetAsync(w + l.off_err, 0, kHeaderBytes, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) {
            ssspmv_plan_destroy(p);
            return record_cuda_error(e);
        }
        launch_partition(row_ptr, m, nnz, l.L, l.ntiles,
                         reinterpret_cast<int32_t *>(w + l.off_tile_offset),
                         reinterpret_cast<uint32_t *>(w + l.off_err),
                         static_cast<cudaStream_t>(stream), partition_method(m, l.ntiles));
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            ssspmv_plan_destroy(p);
            return record_cuda_error(e);
        }
    }
    *out = p;
    return SSSPMV_OK;
}

int ssspmv_plan_execute(ssspmv_plan *p, const int32_t *col_idx, const void *val, const void *x,
                        void *y, void *timer, void *stream)
{
    if (!p) return SSSPMV_EINVAL;
    const Prec *pr = prec_for(p->val_bytes);
    if (!pr) return SSSPMV_EUNSUPPORTED;
    int rc = check_csr_args(p->m, p->n, p->nnz, p->row_ptr, col_idx, val, x, y);
    if (rc) return rc;
    if (p->m == 0) return SSSPMV_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda_error(e);
    if (dev != p->dev) return SSSPMV_EINVAL;  // a plan belongs to the device it was made on
    Call c;
    c.m = p->m;
    c.n = p->n;
    c.nnz = p->nnz;
    c.row_ptr = p->row_ptr;
    c.col = col_idx;
    c.val = val;
    c.x = x;
    c.y = y;
    c.lay = p->lay;
    c.ws = static_cast<unsigned char *>(p->ws);
    c.stream = static_cast<cudaStream_t>(stream);
    c.ev = timer ? timer_next_slot(static_cast<ssspmv_timer *>(timer)) : nullptr;
    c.exact = p->exact;
    c.block_warps = p->block_warps;
    c.skip_partition = 1;
    return pr->run(c);
}

int ssspmv_plan_workspace(const ssspmv_plan *p, void **ptr, size_t *bytes)
{
    if (!p) return SSSPMV_EINVAL;
    if (ptr) *ptr = p->ws;
    if (bytes) *bytes = p->ws_bytes;
    return SSSPMV_OK;
}

void ssspmv_plan_destroy(ssspmv_plan *p)
{
    if (!p) return;
    if (p->owns_ws && p->ws) cudaFree(p->ws);
    delete p;
}

int ssspmv_cached_workspace(void *stream, void **ptr, size_t *bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda_error(e);
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    for (auto &w : g_ws)
        if (w.dev == dev && w.stream == stream && w.ptr) {
            if (ptr) *ptr = w.ptr;
            if (bytes) *bytes = w.bytes;
            return SSSPMV_OK;
        }
    if (ptr) *ptr = nullptr;
    if (bytes) *bytes = 0;
    return SSSPMV_EWORKSPACE;
}

void ssspmv_release_workspaces(void)
{
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &w : g_ws) {
        if (!w.base) continue;
        cudaSetDevice(w.dev);
        cudaFree(w.base);  // waits for the work still using it
    }
    cudaSetDevice(cur);
    g_ws.clear();
}

int ssspmv_csr_f64_axpby(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                         const int32_t *col_idx, const double *val, const double *x, double *y,
                         double alpha, double beta, const ssspmv_opts *opts, void *workspace,
                         size_t ws_bytes, void *stream)
{
    return run_call(8, m, n, nnz, row_ptr, col_idx, val, x, y, opts, workspace, ws_bytes, stream,
                    nullptr, nullptr, nullptr, alpha, beta, 1);
}

int ssspmv_plan_execute_axpby(ssspmv_plan *p, const int32_t *col_idx, const void *val,
                              const void *x, void *y, double alpha, double beta, void *timer,
                              void *stream)
{
    if (!p) return SSSPMV_EINVAL;
    if (p->val_bytes != 8) return SSSPMV_EUNSUPPORTED;
    const Prec *pr = prec_for(p->val_bytes);
    int rc = check_csr_args(p->m, p->n, p->nnz, p->row_ptr, col_idx, val, x, y);
    if (rc) return rc;
    if (p->m == 0) return SSSPMV_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda_error(e);
    if (dev != p->dev) return SSSPMV_EINVAL;
    Call c;
    c.m = p->m;
    c.n = p->n;
    c.nnz = p->nnz;
    c.row_ptr = p->row_ptr;
    c.col = col_idx;
    c.val = val;
    c.x = x;
    c.y = y;
    c.lay = p->lay;
    c.ws = static_cast<unsigned char *>(p->ws);
    c.stream = static_cast<cudaStream_t>(stream);
    c.ev = timer ? timer_next_slot(static_cast<ssspmv_timer *>(timer)) : nullptr;
    c.exact = 1;  // see run_call
    c.block_warps = p->block_warps;
    c.skip_partition = 1;
    c.alpha = alpha;
    c.beta = beta;
    c.axpby = 1;
    return pr->run(c);
}

int ssspmv_csr_f64_debug(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                         const int32_t *col_idx, const double *val, const double *x, double *y,
                         const ssspmv_opts *opts, void *workspace, size_t ws_bytes, void *stream,
                         int32_t *tile_offset, uint32_t *desc, uint32_t *tile_info,
                         int32_t *sync_idx, double *y_spec)
{
    if (!workspace) return SSSPMV_EWORKSPACE;  // the artefacts are read back from it
    Layout l;
    int rc = run_call(8, m, n, nnz, row_ptr, col_idx, val, x, y, opts, workspace, ws_bytes, stream,
                      desc, y_spec, &l);
    if (rc) return rc;
    if (m == 0) return SSSPMV_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaError_t e = cudaSuccess;
    if (tile_offset && e == cudaSuccess)
        e = cudaMemcpyAsync(tile_offset, ws + l.off_tile_offset,
                            sizeof(int32_t) * (size_t)(l.ntiles + 1), cudaMemcpyDeviceToDevice, s);
    if (tile_info && l.ntiles > 0 && e == cudaSuccess)
        e = cudaMemcpyAsync(tile_info, ws + l.off_tile_info, sizeof(uint32_t) * (size_t)l.ntiles,
                            cudaMemcpyDeviceToDevice, s);
    if (sync_idx && l.nbunches > 0 && e == cudaSuccess)
        e = cudaMemcpyAsync(sync_idx, ws + l.off_sync_idx, sizeof(int32_t) * (size_t)l.nbunches,
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return record_cuda_error(e);
    uint32_t bits = 0;
    rc = ssspmv_device_status(workspace, ws_bytes, stream, 0, &bits);
    if (rc) return rc;
    return bits ? SSSPMV_EDEVICE : SSSPMV_OK;
}

int ssspmv_device_status(void *workspace, size_t ws_bytes, void *stream, int clear,
                         uint32_t *bits)
{
    if (!workspace || ws_bytes < 16) return SSSPMV_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && clear) e = cudaMemsetAsync(workspace, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return record_cuda_error(e);
    if (bits) *bits = h;
    return SSSPMV_OK;
}

size_t ssspmv_host_buffer_bytes(int32_t m, int32_t n, int32_t nnz, const ssspmv_opts *opts)
{
    if (m < 0 || n < 0 || nnz < 0) return 0;
    size_t ws = ssspmv_workspace_bytes(m, nnz, 8, opts);
    if (ws == 0) return 0;
    size_t o = 0;
    o = align256(o + sizeof(int32_t) * ((size_t)m + 1));
    o = align256(o + sizeof(int32_t) * (size_t)nnz);
    o = align256(o + sizeof(double) * (size_t)nnz);
    o = align256(o + sizeof(double) * (size_t)n);
    o = align256(o + sizeof(double) * (size_t)m);
    return o + ws;
}

int ssspmv_csr_f64_host(int32_t m, int32_t n, int32_t nnz, const int32_t *host_row_ptr,
                        const int32_t *host_col_idx, const double *host_val,
                        const double *host_x, double *host_y, const ssspmv_opts *opts,
                        void *dev_buffer, size_t dev_bytes, void *stream)
{
    int rc = check_csr_args(m, n, nnz, host_row_ptr, host_col_idx, host_val, host_x, host_y);
    if (rc && rc != SSSPMV_EINVAL) return rc;
    if (m < 0 || n < 0 || nnz < 0 || (m == 0 && nnz != 0)) return SSSPMV_EINVAL;
    if (m > 0 && (!host_row_ptr || !host_y)) return SSSPMV_EINVAL;
    if (nnz > 0 && (!host_col_idx || !host_val || !host_x || n == 0)) return SSSPMV_EINVAL;
    if (m == 0) return SSSPMV_OK;
    const size_t need = ssspmv_host_buffer_bytes(m, n, nnz, opts);
    if (need == 0) return SSSPMV_EINVAL;
    if (!dev_buffer || dev_bytes < need || ((uintptr_t)dev_buffer & 255u))
        return SSSPMV_EWORKSPACE;
    unsigned char *p = static_cast<unsigned char *>(dev_buffer);
    size_t o = 0;
    int32_t *d_rp = reinterpret_cast<int32_t *>(p + o);
    o = align256(o + sizeof(int32_t) * ((size_t)m + 1));
    int32_t *d_col = reinterpret_cast<int32_t *>(p + o);
    o = align256(o + sizeof(int32_t) * (size_t)nnz);
    double *d_val = reinterpret_cast<double *>(p + o);
    o = align256(o + sizeof(double) * (size_t)nnz);
    double *d_x = reinterpret_cast<double *>(p + o);
    o = align256(o + sizeof(double) * (size_t)n);
    double *d_y = reinterpret_cast<double *>(p + o);
    o = align256(o + sizeof(double) * (size_t)m);
    void *ws = p + o;
    const size_t ws_bytes = dev_bytes - o;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(d_rp, host_row_ptr, sizeof(int32_t) * ((size_t)m + 1),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(d_col, host_col_idx, sizeof(int32_t) * (size_t)nnz,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(d_val, host_val, sizeof(double) * (size_t)nnz, cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(d_x, host_x, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return record_cuda_error(e);
    rc = ssspmv_csr_f64(m, n, nnz, d_rp, d_col, d_val, d_x, d_y, opts, ws, ws_bytes, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(host_y, d_y, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return record_cuda_error(e);
    return SSSPMV_OK;
}

int ssspmv_validate_csr(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, void *scratch, void *stream)
{
    if (m < 0 || n < 0 || nnz < 0 || !scratch) return SSSPMV_EINVAL;
    if (m > 0 && !row_ptr) return SSSPMV_EINVAL;
    if (nnz > 0 && !col_idx) return SSSPMV_EINVAL;
    if (m == 0) return nnz == 0 ? SSSPMV_OK : SSSPMV_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *bad = static_cast<uint32_t *>(scratch);
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return record_cuda_error(e);
    validate_kernel<<<4 * device_sm_count(), 256, 0, s>>>(m, n, nnz, row_ptr, col_idx, bad);
    e = cudaGetLastError();
    uint32_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return record_cuda_error(e);
    return h ? SSSPMV_EINVAL : SSSPMV_OK;
}

}  // extern "C"
