// segsum.cuh -- the three kernels of CSR SpMV by speculative segmented sum
// (Liu & Vinter, Sec. 3 and Algorithm 1), written for sm_103a.
//
//   (a) partition_kernel   tile_offset[t] = max{r : row_ptr[r] <= b_t}
//   (b) segsum_kernel      per tile: on-chip row-start descriptor from row_ptr,
//                          x gathers, FMA accumulation per segment, transmitter
//                          carried between the tiles of a bunch, speculative
//                          stores y[tile_offset[t] + s], synchronizer records
//   (c) calibrate_kernel   synchronizer sums, re-arrangement of dirty tiles,
//                          zeroing of empty rows
//
// Tile t holds the nonzeros [b_t, b_{t+1}), b_t = min(t*L, nnz), L = 32*W.
// A warp is the paper's thread-bunch and owns S consecutive tiles; lane l of
// the warp owns the W consecutive entries [l*W, (l+1)*W) of each tile (the
// W x T tile of Sec. 3.1).  W is odd, so lane-strided shared-memory reads of
// a tile are free of bank conflicts without padding, and 32*W entries of 4 or
// 8 bytes are still a multiple of 16 bytes for the bulk copies.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "layout.h"
#include "ptx.cuh"

namespace ssspmv {

// ---------------------------------------------------------------------------
// precision traits

struct F64 {
    // most warps per SM that the registers allow at tile width W
    static constexpr int max_warps(int) { return 32; }  // shared memory decides
    // scan the rows of a tile over many rows before its gathers (measured:
    // R-MAT scale 22 kernel (b) 362 -> 350 us; the FP32 forms lose 2-3%)
    static constexpr bool kEarlyLongScan = true;
    static constexpr int kShortRowWarps = 14;  // short rows: keep L1 for the gathers (measured)
    using val_t = double;
    using x_t = double;
    using y_t = double;
    using acc_t = double;
    __device__ static __forceinline__ acc_t zero() { return 0.0; }
    __device__ static __forceinline__ acc_t fma(val_t v, x_t x, acc_t a) { return __fma_rn(v, x, a); }
    __device__ static __forceinline__ acc_t add(acc_t a, acc_t b) { return __dadd_rn(a, b); }
    __device__ static __forceinline__ y_t out(acc_t a) { return a; }
    __device__ static __forceinline__ double to_f64(acc_t a) { return a; }
    __device__ static __forceinline__ acc_t shfl_up(acc_t a, int d)
    {
        return __shfl_up_sync(FULL, a, d);
    }
    __device__ static __forceinline__ acc_t shfl(acc_t a, int src)
    {
        return __shfl_sync(FULL, a, src);
    }
    __device__ static __forceinline__ x_t gather(const x_t *x, int32_t c, uint64_t pol)
    {
        return ldg_keep(x + c, pol);
    }
};

// FP32 accumulation carried as an unevaluated sum s + c: each product is
// split exactly by TwoProduct (fused multiply-add) and added with TwoSum
// (Knuth), the Dot2 scheme of Ogita, Rump and Oishi (SIAM J. Sci. Comput.
// 2005) in single precision.
struct CompF32 {
    float s, c;
};

__device__ __forceinline__ CompF32 comp_add(CompF32 a, CompF32 b)
{
    const float s = __fadd_rn(a.s, b.s);
    const float z = __fadd_rn(s, -a.s);
    const float t = __fadd_rn(__fadd_rn(a.s, -__fadd_rn(s, -z)), __fadd_rn(b.s, -z));
    return CompF32{s, __fadd_rn(__fadd_rn(a.c, b.c), t)};
}

__device__ __forceinline__ CompF32 comp_fma(float v, float x, CompF32 a)
{
    const float p = __fmul_rn(v, x);
    const float e = __fmaf_rn(v, x, -p);        // v*x - p exactly
    const float s = __fadd_rn(a.s, p);
    const float z = __fadd_rn(s, -a.s);
    const float t = __fadd_rn(__fadd_rn(a.s, -__fadd_rn(s, -z)), __fadd_rn(p, -z));
    return CompF32{s, __fadd_rn(a.c, __fadd_rn(t, e))};
}

template <class V>
struct CompF32Traits {
    // FP32 values: 24 warps (80 registers per thread, no spills at W = 15);
    // BF16 values: 24 at W = 15 (80 registers, no spills), 20 for longer
    // tiles, whose widened values need 96 registers
    static constexpr int max_warps(int W)
    {
        return (std::is_same<V, float>::value || W <= 15) ? 24 : 20;
    }
    static constexpr int kBatchMaxWarps = 20;  // the batched kernel needs more registers
    static constexpr bool kEarlyLongScan = false;  // see F64
    static constexpr int kShortRowWarps = 16;  // short rows: keep L1 for the gathers (measured)
    using val_t = V;
    using x_t = float;
    using y_t = float;
    using acc_t = CompF32;
    __device__ static __forceinline__ float widen(float v) { return v; }
    __device__ static __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ acc_t zero() { return CompF32{0.f, 0.f}; }
    __device__ static __forceinline__ acc_t fma(val_t v, x_t x, acc_t a)
    {
        return comp_fma(widen(v), x, a);
    }
    __device__ static __forceinline__ acc_t add(acc_t a, acc_t b) { return comp_add(a, b); }
    __device__ static __forceinline__ y_t out(acc_t a) { return __fadd_rn(a.s, a.c); }
    __device__ static __forceinline__ double to_f64(acc_t a) { return (double)a.s + (double)a.c; }
    __device__ static __forceinline__ acc_t shfl_up(acc_t a, int d)
    {
        return CompF32{__shfl_up_sync(FULL, a.s, d), __shfl_up_sync(FULL, a.c, d)};
    }
    __device__ static __forceinline__ acc_t shfl(acc_t a, int src)
    {
        return CompF32{__shfl_sync(FULL, a.s, src), __shfl_sync(FULL, a.c, src)};
    }
    __device__ static __forceinline__ x_t gather(const x_t *x, int32_t c, uint64_t pol)
    {
        return ldg_keep(x + c, pol);
    }
};

using F32C = CompF32Traits<float>;           // FP32 val, x, y
using BF16C = CompF32Traits<__nv_bfloat16>;  // BF16 val, FP32 x, y

// ---------------------------------------------------------------------------
// kernel (a): partition (Sec. 3.2: binary search of the tile boundaries on
// row_ptr, returning the rightmost match).  One thread per boundary.

// Thread 0 also clears the workspace's device error word for this call.
// method 0 = binary search per boundary, 1 = row-parallel scatter (same result).
void launch_partition(const int32_t *row_ptr, int32_t m, int32_t nnz, int32_t L, int64_t ntiles,
                      int32_t *tile_offset, uint32_t *err, cudaStream_t stream, int method);
// the method used when the caller does not choose (the cheaper one)
int partition_method(int32_t m, int64_t ntiles);

// ---------------------------------------------------------------------------
// shared-memory layout of one warp in kernel (b)

template <class P, int W>
struct WarpSmem {
    static constexpr int L = 32 * W;
    static constexpr int VAL_BYTES = L * (int)sizeof(typename P::val_t);
    static constexpr int COL_BYTES = L * 4;
    static constexpr int VAL_REGION = (VAL_BYTES + 15) & ~15;
    static constexpr int STAGE_BYTES = ((VAL_REGION + COL_BYTES) + 127) & ~127;
    static constexpr int STAGES = 2;
    static constexpr int BAR_OFF = STAGES * STAGE_BYTES;
    static constexpr int DESC_OFF = BAR_OFF + STAGES * 8;
    static constexpr int DESC_WORDS = W + 1;  // one spare word for 64-bit windows
    static constexpr int SLOT_OFF = (DESC_OFF + DESC_WORDS * 4 + 15) & ~15;
    // slot: the bunch-first partial, the transmitter, the warp's schedule
    static constexpr int BYTES = (SLOT_OFF + 48 + 127) & ~127;
};

// Warps per block (B) and blocks per SM maximising resident warps per SM for
// a per-warp shared-memory footprint (228 KB per SM, 227 KB per block, 1 KB
// reserved per block) under a register budget of max_warps warps per SM.
struct BlockShape {
    int B, blocks;
};

constexpr BlockShape pick_block_shape(int warp_bytes, int max_warps)
{
    BlockShape best{1, 1};
    int best_w = 0;
    for (int b = 1; b <= 32 && b <= max_warps; ++b) {
        const long blk = (long)b * warp_bytes;
        if (blk > 232448) break;
        int per_sm = (int)(233472 / (blk + 1024));
        if (per_sm * b > max_warps) per_sm = max_warps / b;
        if (per_sm < 1) continue;
        const int w = per_sm * b;
        if (w >= best_w) {
            best_w = w;
            best = BlockShape{b, per_sm};
        }
    }
    return best;
}

// One matrix of a batch as the kernels see it: the caller's arrays plus its
// place in the batch's global tile, bunch and row numbering (filled on the
// device from the caller's descriptors by the batch set-up kernel).
struct BatchMat {
    const void *val;
    const int32_t *col;
    const int32_t *row_ptr;
    const void *x;
    void *y;
    int32_t m, nnz;
    int32_t tile_base;   // global index of its first tile
    int32_t bunch_base;  // global index of its first bunch
    int32_t ntiles;      // its tile count
    int32_t row_base;    // global index of its first row
};
static_assert(sizeof(BatchMat) == kBatchMatBytes, "BatchMat is one 64-byte record");

template <class T>
__device__ __forceinline__ T *ldg_ptr(T *const *p)
{
    return reinterpret_cast<T *>(__ldg(reinterpret_cast<const unsigned long long *>(p)));
}

struct SegsumArgs {
    const int32_t *row_ptr;
    const int32_t *col;
    const void *val;
    const void *x;
    void *y;
    const int32_t *tile_offset;
    uint32_t *tile_info;
    int32_t *sync_idx;
    void *sync_val;
    void *tail_val;
    int32_t *tail_flag;
    uint32_t *err;
    uint32_t *ticket;    // bunch ticket counter, zero at launch
    // dirty tiles left speculative are appended here for kernel (c) (the
    // paper's speculator and dirty counter); the count is zero at launch
    uint32_t *dirty_count = nullptr;
    int32_t *dirty_list = nullptr;
    // nullable: nonzero when kernel (a) saw a run of 32 empty rows (tiles
    // over thousands of rows may follow): a smaller static share then
    const uint32_t *spread = nullptr;
    uint32_t *dbg_desc;  // nullable
    int32_t m;
    int32_t nnz;
    int64_t ntiles;
    int64_t nbunches;
    int32_t S;
    // batches only: the matrices, the matrix of every global bunch, and the
    // batch totals {tiles, bunches} (all written on the device)
    const BatchMat *mats = nullptr;
    const int32_t *bunch_mat = nullptr;
    const int32_t *totals = nullptr;
    // y = alpha A x + beta y (exact stores only; off: y = A x)
    double alpha = 1.0, beta = 0.0;
    int32_t axpby = 0;
};

// the value a final store of row `row` writes: v, or alpha v + beta y[row]
// (y is not read when beta is 0)
template <class Y>
__device__ __forceinline__ Y scaled_store_value(const Y *y, int64_t row, Y v, double alpha,
                                                double beta, int32_t on)
{
    if (!on) return v;
    const double av = alpha * (double)v;
    return (Y)(beta != 0.0 ? fma(beta, (double)y[row], av) : av);
}

// tile_info layout: bit 31 dirty, bit 30 dirty and resolved by kernel (b),
// bits 0..29 number of segments
constexpr uint32_t kInfoDirty = 0x80000000u;
constexpr uint32_t kInfoResolved = 0x40000000u;
constexpr uint32_t kInfoSegMask = 0x3fffffffu;

// dirty tiles over more rows than this are re-arranged by a whole block in
// kernel (c), which keeps up to kLongListCap of them at a time
constexpr int32_t kLongRepairRows = 1024;
constexpr int kLongListCap = 512;

// ---------------------------------------------------------------------------
// descriptor scan of rows [rb0, stop] for tiles over many (mostly empty) rows,
// CH chunks of 32 rows per round trip.  A run of empty rows shares one row
// pointer: only its last row (the non-empty row, or `stop`) sets the bit, so
// the atomics do not pile up on one word.  Kept out of line: the call is rare
// and the loop then keeps its loads in flight with registers of its own.
// Called with CH = 16 before a tile's gathers are issued (no gathered x held
// in registers), with CH = 4 after them (more would spill the FP64 kernel's
// registers).  Returns bit 0: an empty row in [rb0, stop); bit 1: row `stop`
// starts inside the tile.  With exact stores (xs) it also writes the
// position-to-row map and zeroes the empty rows.
template <class Y, int CH>
__device__ __noinline__ uint32_t scan_rows_long(const int32_t *__restrict__ row_ptr, int32_t m,
                                                int32_t rb0, int32_t stop, int32_t b, int32_t len,
                                                uint32_t *desc, int32_t *rowmap, Y *y,
                                                double alpha, double beta, int32_t axpby, bool xs)
{
    const int lane = threadIdx.x & 31;
    const int32_t e = b + len;
    uint32_t flags = 0;
    for (int32_t rb = rb0; rb <= stop; rb += 32 * CH) {
        int32_t prs[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int32_t r = rb + 32 * u + lane;
            prs[u] = __ldg(row_ptr + (r < m ? r : m));
        }
        int32_t tail = 0;
        if (lane == 31 && rb + 32 * CH - 1 < stop) tail = __ldg(row_ptr + rb + 32 * CH);
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int32_t r = rb + 32 * u + lane;
            const int32_t pr = prs[u];
            const int32_t nlead = __shfl_sync(FULL, prs[u < CH - 1 ? u + 1 : CH - 1], 0);
            int32_t nx = __shfl_down_sync(FULL, pr, 1);
            if (lane == 31) nx = (u < CH - 1) ? nlead : tail;
            if (r <= stop) {
                const int32_t k = pr - b;
                if (k >= 0 && k < len && (r == stop || nx != pr))
                    atomicOr(&desc[k >> 5], 1u << (k & 31));
                if (r < stop) {
                    if (nx == pr) {
                        flags |= 1u;
                        if (xs) y[r] = scaled_store_value(y, r, Y(0), alpha, beta, axpby);
                    } else if (xs && k > 0) {
                        rowmap[k] = r;
                    }
                }
                if (r == stop && pr < e) flags |= 2u;
            }
        }
    }
    return flags;
}

// ---------------------------------------------------------------------------
// kernel (b): a thread-bunch (warp) processes S consecutive tiles, carrying the
// transmitter from tile to tile.  Bunches go to a persistent grid of warps:
// warp g first streams a contiguous range of bunches (3/4 of all bunches are
// split evenly this way, so the copy stream of a warp runs through memory in
// order), then takes the remaining bunches one at a time from a ticket
// counter, which evens out bunches that cost more (tiles over many rows).
// Tickets run from the last bunch backwards: the sparse end of a matrix
// (tiles over many, mostly empty rows) is started first, not left to the
// tail of the launch.

template <class P, int W, int B, int MINB, bool EXACT, bool BATCHED = false>
__global__ void __launch_bounds__(B * 32, MINB) segsum_kernel(const SegsumArgs a)
{
    using V = typename P::val_t;
    using X = typename P::x_t;
    using Y = typename P::y_t;
    using A = typename P::acc_t;
    using SM = WarpSmem<P, W>;
    constexpr int L = SM::L;
    constexpr int STAGES = SM::STAGES;
    static_assert(W % 2 == 1 && W <= 31, "W must be odd and at most 31");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + warp * SM::BYTES;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + SM::BAR_OFF);
    uint32_t *desc = reinterpret_cast<uint32_t *>(base + SM::DESC_OFF);
    A *slot_f = reinterpret_cast<A *>(base + SM::SLOT_OFF);           // bunch-first partial
    A *slot_carry = reinterpret_cast<A *>(base + SM::SLOT_OFF + 16);  // transmitter

    // tiles, bunches, rows and positions all fit in 32 bits (the host
    // rejects m or nnz within 256 of the int32 limit)
    // a batch is one global sequence of tiles and bunches; its totals are
    // known on the device only
    const int32_t nb = BATCHED ? __ldg(a.totals + 1) : (int32_t)a.nbunches;
    const int32_t ntiles = BATCHED ? __ldg(a.totals) : (int32_t)a.ntiles;
    // blocks may be launched with fewer than B warps (more L1 per warp)
    const int32_t bw = (int32_t)(blockDim.x >> 5);
    const int32_t nwarps = (int32_t)gridDim.x * bw;
    const int32_t g = (int32_t)blockIdx.x * bw + warp;
    if (g >= nb) return;
    // static share: bunches [g*Q, g*Q + Q) (3/4 of the bunches in all); the
    // bunches from nwarps*Q on are handed out by ticket, the last first.
    // When kernel (a) flags runs of empty rows, a bunch may cost as much as a
    // whole static share, so only the first third of each share is kept (at
    // least one bunch) and the rest of the shares joins the ticket pool
    // behind the end of the matrix; the first bunch of a warp is the same
    // either way
    int32_t Q = (int32_t)((3 * (int64_t)nb) / (4 * (int64_t)nwarps));
    if (Q < 1) Q = 1;
    const int32_t dyn_base = nwarps * Q;
    int32_t cur = g * Q;
    int32_t static_end = cur + Q;  // set again once kernel (a) has finished
    // {Q, gap}, gap being the bunches of each share given to the pool: read
    // from the warp's shared slot once the pool's tail part is used up
    volatile int32_t *sched = reinterpret_cast<volatile int32_t *>(base + SM::SLOT_OFF + 32);
    if (lane == 0) {
        sched[0] = Q;
        sched[1] = 0;
    }
    __syncwarp();

    // the matrix of the current bunch (in a batch: reloaded per bunch);
    // tbase is the global index of its first tile, shift its index in the
    // batch (its tile offsets start at global position tbase + shift)
    const V *__restrict__ val = static_cast<const V *>(a.val);
    const X *__restrict__ x = static_cast<const X *>(a.x);
    Y *__restrict__ y = static_cast<Y *>(a.y);
    const int32_t *__restrict__ row_ptr = a.row_ptr;
    const int32_t *__restrict__ col = a.col;
    int32_t nnz = a.nnz, mrows = a.m, tbase = 0, shift = 0;
    const int32_t S = a.S;
    auto load_matrix = [&](int32_t mi) {
        if constexpr (BATCHED) {
            const BatchMat *mm = a.mats + mi;
            val = static_cast<const V *>(ldg_ptr(&mm->val));
            x = static_cast<const X *>(ldg_ptr(&mm->x));
            y = static_cast<Y *>(ldg_ptr(const_cast<void *const *>(&mm->y)));
            row_ptr = ldg_ptr(&mm->row_ptr);
            col = ldg_ptr(&mm->col);
            nnz = __ldg(&mm->nnz);
            mrows = __ldg(&mm->m);
            tbase = __ldg(&mm->tile_base);
            shift = mi;
        }
    };
    auto mat_of = [&](int32_t bb) -> int32_t {
        if constexpr (BATCHED) return __ldg(a.bunch_mat + bb);
        else return 0;
    };
    // global index of bunch bb's first tile, and one past its last
    auto first_tile = [&](int32_t bb, int32_t mi) -> int32_t {
        if constexpr (BATCHED)
            return __ldg(&a.mats[mi].tile_base) + (bb - __ldg(&a.mats[mi].bunch_base)) * S;
        else return bb * S;
    };

    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();

    auto bunch_end = [&](int32_t bb, int32_t mi) -> int32_t {
        if constexpr (BATCHED) {
            const int32_t f = first_tile(bb, mi);
            const int32_t e = __ldg(&a.mats[mi].tile_base) + __ldg(&a.mats[mi].ntiles);
            return f + S < e ? f + S : e;
        } else {
            return (bb * S + S < ntiles) ? bb * S + S : ntiles;
        }
    };
    int32_t nxt = -1;  // the warp's next bunch, once known (warp-uniform)
    int32_t ni = 0;    // its matrix
    uint32_t tk = 0;   // lane 0: a ticket requested ahead of its use
    bool tk_pending = false;
    auto request_ticket = [&]() {  // the atomic's round trip overlaps the bunch
        if (nxt >= 0 || tk_pending || cur + 1 < static_end) return;
        if (lane == 0) tk = atomicAdd(a.ticket, 1u);
        tk_pending = true;
    };
    auto claim_next = [&]() {
        if (nxt >= 0) return;
        if (cur + 1 < static_end) {
            nxt = cur + 1;
            if (BATCHED && nxt < nb) ni = mat_of(nxt);
            return;
        }
        request_ticket();
        tk_pending = false;
        const int32_t k = (int32_t)__shfl_sync(FULL, tk, 0);
        // the static share is over for good: a bunch of the pool (a share's
        // gap may lie below this share) is never continued as if static
        static_end = 0;
        if (k < nb - dyn_base) {
            nxt = nb - 1 - k;
        } else {
            // the j-th bunch of the shares' gaps (share g' gives up its last
            // gap bunches): j / gap through a float reciprocal and one
            // correction (exact: j and gap are below 2^24), which costs
            // fewer registers than an integer division
            const int32_t j = k - (nb - dyn_base), gap = sched[1];
            nxt = nb;
            if (gap > 0 && j < (int32_t)gridDim.x * (int32_t)(blockDim.x >> 5) * gap) {
                int32_t w = __float2int_rz((float)j * __frcp_rn((float)gap));
                if ((w + 1) * gap <= j) ++w;
                if (w * gap > j) --w;
                const int32_t q = sched[0];
                nxt = w * q + (q - gap) + (j - w * gap);
            }
        }
        if (BATCHED && nxt < nb) ni = mat_of(nxt);
    };

    auto stage_ptr = [&](uint32_t s) { return base + s * SM::STAGE_BYTES; };
    // bulk copies of tile tt (of matrix mi) into stage s (lane 0 only)
    auto issue = [&](int32_t tt, uint32_t s, int32_t mi) {
        const V *vsrc = val;
        const int32_t *csrc = col;
        int32_t nz = nnz, tb = 0;
        if constexpr (BATCHED) {
            const BatchMat *mm = a.mats + mi;
            vsrc = static_cast<const V *>(ldg_ptr(&mm->val));
            csrc = ldg_ptr(&mm->col);
            nz = __ldg(&mm->nnz);
            tb = __ldg(&mm->tile_base);
        }
        const int32_t b = (tt - tb) * L;
        const int32_t len = (nz - b < L) ? nz - b : L;
        const uint32_t vb = ((uint32_t)len * (uint32_t)sizeof(V)) & ~15u;
        const uint32_t cb = ((uint32_t)len * 4u) & ~15u;
        mbar_arrive_expect_tx(&bar[s], vb + cb);
        if (vb) bulk_g2s(stage_ptr(s), vsrc + b, vb, &bar[s], pol_stream);
        if (cb) bulk_g2s(stage_ptr(s) + SM::VAL_REGION, csrc + b, cb, &bar[s], pol_stream);
    };
    // the copy stream runs at most STAGES tiles ahead, into at most the next
    // bunch (warp-uniform: every lane calls it)
    int32_t ci = mat_of(cur);  // the current bunch's matrix
    load_matrix(ci);
    int32_t iss_b = cur, iss_i = ci, iss_t = first_tile(cur, ci);
    uint32_t q_iss = 0, q_con = 0;  // tiles issued / consumed by this warp
    auto issue_next = [&]() {
        if (iss_b >= nb) return;
        if (iss_t >= bunch_end(iss_b, iss_i)) {
            if (iss_b != cur) return;
            claim_next();
            iss_b = nxt;
            iss_i = ni;
            if (iss_b >= nb) return;
            iss_t = first_tile(nxt, ni);
        }
        if (lane == 0) {
            fence_proxy_async_smem();
            issue(iss_t, q_iss % STAGES, iss_i);
        }
        ++q_iss;
        ++iss_t;
    };

    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if constexpr (!BATCHED) {
        // the warp's first tile is input only (no ticket, no tile offset):
        // its copy is under way while kernel (a) finishes; nothing kernel (a)
        // writes is read before grid_dep_wait()
        issue_next();
        grid_dep_wait();
        grid_dep_trigger();
        // kernel (a)'s schedule flag (a share of one bunch stays whole: the
        // flag is not read then); applied before the first claim
        if (Q >= 2 && a.spread != nullptr && *(volatile const uint32_t *)a.spread != 0u) {
            const int32_t qs = Q >= 3 ? Q / 3 : 1;
            static_end = cur + qs;
            if (lane == 0) sched[1] = Q - qs;
            __syncwarp();
        }
        for (int s = 1; s < STAGES; ++s) issue_next();
    } else {
        for (int s = 0; s < STAGES; ++s) issue_next();
    }

    // boundary rows and the first row-pointer chunk of the next tile, loaded
    // one tile ahead (rows past m read row_ptr[m])
    int32_t start = __ldg(a.tile_offset + first_tile(cur, ci) + shift);
    int32_t stop = __ldg(a.tile_offset + first_tile(cur, ci) + shift + 1);
    auto rp_at = [&](int32_t r) { return __ldg(row_ptr + (r < mrows ? r : mrows)); };
    int32_t pr_chunk = rp_at(start + lane);
    int32_t pr_chunk2 = rp_at(start + 32 + lane);

    while (true) {
        request_ticket();
        const int32_t t0 = first_tile(cur, ci), t1 = bunch_end(cur, ci);
        const int32_t rF = start;  // the bunch's first row
        A carry = P::zero();
        A G = P::zero();
        bool hasG = false;

        for (int32_t t = t0; t < t1; ++t) {
            const uint32_t s = q_con % STAGES;
            const uint32_t par = (q_con / STAGES) & 1u;
            const int32_t b = (t - tbase) * L;  // the tile's entries [b, e) of its matrix
            const int32_t len = (nnz - b < L) ? nnz - b : L;
            const int32_t e = b + len;

            // ---- prefetch the next tile's rows (the next bunch's first tile
            // after the last one)
            int32_t start_nx = stop, stop_nx = 0, pr_nx = 0, pr_nx2 = 0;
            if (t + 1 < t1) {
                stop_nx = __ldg(a.tile_offset + t + 2 + shift);
                pr_nx = rp_at(start_nx + lane);
                pr_nx2 = rp_at(start_nx + 32 + lane);
            } else {
                claim_next();
                if (nxt < nb) {
                    const int32_t ft = first_tile(nxt, ni) + (BATCHED ? ni : 0);
                    start_nx = __ldg(a.tile_offset + ft);
                    stop_nx = __ldg(a.tile_offset + ft + 1);
                    const int32_t *rp = row_ptr;
                    int32_t mm = mrows;
                    if constexpr (BATCHED) {
                        rp = ldg_ptr(&a.mats[ni].row_ptr);
                        mm = __ldg(&a.mats[ni].m);
                    }
                    const int32_t r1 = start_nx + lane, r2 = start_nx + 32 + lane;
                    pr_nx = __ldg(rp + (r1 < mm ? r1 : mm));
                    pr_nx2 = __ldg(rp + (r2 < mm ? r2 : mm));
                }
            }

            // ---- wait for this tile's val/col
            unsigned char *st = stage_ptr(s);
            const V *vs = reinterpret_cast<const V *>(st);
            const int32_t *cs = reinterpret_cast<const int32_t *>(st + SM::VAL_REGION);
            if (!mbar_wait_bounded(&bar[s], par)) {
                if (lane == 0) atomicOr(a.err, SSSPMV_DEV_TIMEOUT);
                // drain the copies still in flight before leaving
                for (uint32_t q = q_con; q < q_iss; ++q)
                    mbar_wait_bounded(&bar[q % STAGES], (q / STAGES) & 1u);
                return;
            }
            if (len < L) {  // ragged last tile: the bulk copies stop at 16-byte multiples
                V *vw = reinterpret_cast<V *>(st);
                int32_t *cw = reinterpret_cast<int32_t *>(st + SM::VAL_REGION);
                const int32_t vdone =
                    (int32_t)((((uint32_t)len * (uint32_t)sizeof(V)) & ~15u) / sizeof(V));
                const int32_t cdone = (int32_t)((((uint32_t)len * 4u) & ~15u) / 4u);
                // entries past len read as val 0, col 0: the loops below then
                // need no bounds checks (adding 0 * x[0] leaves every sum as is)
                for (int32_t k = vdone + lane; k < L; k += 32) vw[k] = (k < len) ? val[b + k] : V(0);
                for (int32_t k = cdone + lane; k < L; k += 32) cw[k] = (k < len) ? col[b + k] : 0;
                __syncwarp();
            }

            // ---- a tile over many rows with speculative FP64 stores: its rows
            // past the first 64 (usually thousands of mostly empty rows at the
            // sparse end of a power-law matrix) are scanned before the gathers
            // are issued, when no gathered x is held in registers, so the scan
            // keeps 16 chunks of row pointers in flight.  (Exact stores scan
            // after the gathers: their row map goes into the column region
            // the gathers read.)
            uint32_t long_flags = 0;
            const bool long_first = P::kEarlyLongScan && !EXACT && start + 64 <= stop;
            if (long_first) {
                if (lane <= W) desc[lane] = 0u;
                __syncwarp();
                long_flags = scan_rows_long<Y, 16>(row_ptr, mrows, start + 64, stop, b, len, desc,
                                                   nullptr, y, a.alpha, a.beta, a.axpby, false);
            }

            // ---- gathers of x for the lane's W entries (Alg. 1 products),
            // issued before the descriptor work so their latency overlaps it
            X xv[W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const int k = lane * W + j;
                xv[j] = P::gather(x, cs[k], pol_keep);
            }

            // ---- segment descriptor built on chip from row_ptr[start..stop]
            // (Sec. 3.2: offsets of the covered row pointers from the
            // boundary; every row start inside the tile, including row
            // `stop`'s) and the empty-row ("dirty") test over [start, stop).
            // With exact stores, a map from tile position to the non-empty
            // row starting there goes into the stage's column region (free
            // once the gathers above are issued) and empty rows are zeroed.
            int32_t *rowmap = reinterpret_cast<int32_t *>(st + SM::VAL_REGION);
            constexpr bool xs = EXACT;
            if (!long_first && lane <= W) desc[lane] = 0u;
            __syncwarp();
            bool dirty = (long_flags & 1u) != 0, cont = (long_flags & 2u) != 0, raw0 = false;
            auto scan_row = [&](int32_t r, int32_t pr, int32_t nx) {
                if (r > stop) return;
                const int32_t k = pr - b;
                // one bit per distinct pointer: set by the last row of a run
                if (k >= 0 && k < len && (r == stop || nx != pr))
                    atomicOr(&desc[k >> 5], 1u << (k & 31));
                if (r < stop) {
                    if (nx == pr) {
                        dirty = true;
                        // r > start: row `start` is never empty
                        if (xs) y[r] = scaled_store_value(y, r, Y(0), a.alpha, a.beta, a.axpby);
                    } else if (xs && k > 0) {
                        rowmap[k] = (int32_t)r;
                    }
                }
                if (r == start && k == 0) raw0 = true;
                if (r == stop && pr < e) cont = true;
            };
            {
                // rows start .. start+63 were loaded one tile ahead
                int32_t nx = __shfl_down_sync(FULL, pr_chunk, 1);
                const int32_t c2 = __shfl_sync(FULL, pr_chunk2, 0);
                if (lane == 31) nx = c2;
                scan_row(start + lane, pr_chunk, nx);
            }
            if (start + 32 <= stop) {
                int32_t nx = __shfl_down_sync(FULL, pr_chunk2, 1);
                if (lane == 31 && start + 63 < stop) nx = rp_at(start + 64);
                scan_row(start + 32 + lane, pr_chunk2, nx);
                if (!long_first && start + 64 <= stop) {  // long row ranges, exact stores
                    const uint32_t f = scan_rows_long<Y, 4>(row_ptr, mrows, start + 64, stop, b,
                                                            len, desc, rowmap, y, a.alpha, a.beta,
                                                            a.axpby, xs);
                    dirty |= (f & 1u) != 0;
                    cont |= (f & 2u) != 0;
                }
            }
            dirty = __any_sync(FULL, dirty);
            cont = __any_sync(FULL, cont);
            raw0 = __any_sync(FULL, raw0);
            __syncwarp();
            const bool resolve = xs && dirty;
            const int bit0 = lane * W;
            const uint64_t win =
                ((uint64_t)desc[(bit0 >> 5) + 1] << 32) | (uint64_t)desc[bit0 >> 5];
            uint32_t hb = (uint32_t)(win >> (bit0 & 31)) & ((1u << W) - 1u);
            // debug export, added to a zeroed buffer: a tile processed twice
            // would show doubled words
            if (a.dbg_desc != nullptr && lane < W) atomicAdd(a.dbg_desc + t * W + lane, desc[lane]);
            if (lane == 0) hb |= 1u;  // each tile opens with a segment (Sec. 3.2)

            // ---- compact indices: exclusive scan of head counts (y_index)
            const int c = __popc(hb);
            const int incl = warp_inclusive_scan(c, lane);
            const int idx0 = incl - c;
            const int nseg = __shfl_sync(FULL, incl, 31);
            const A cin = (raw0 || t == t0) ? P::zero() : carry;  // transmitter

            // segment sidx goes to the synchronizer slot (the bunch's first
            // segment), to its speculative row start + sidx (Alg. 1), or --
            // exact stores on a dirty tile -- to the row that starts at its
            // head position hpos (read only then)
            auto emit = [&](int sidx, A v, int hpos) {
                if (sidx == 0 && start == rF) {
                    *slot_f = v;
                } else {
                    int32_t row = start + sidx;
                    if (resolve) row = hpos <= 0 ? start : rowmap[hpos < L ? hpos : 0];
                    if (row >= 0 && row < mrows) {
                        if constexpr (EXACT)
                            y[row] = scaled_store_value(y, row, P::out(v), a.alpha, a.beta, a.axpby);
                        else
                            y[row] = P::out(v);
                    }
                    else atomicOr(a.err, SSSPMV_DEV_RANGE);
                }
            };

            // ---- per-lane sequential segmented sum, one FMA per entry in one
            // chain (the FP64 pipe, not the chain's latency, sets the pace)
            // head positions, where exact stores need them, come from hb: the
            // lane's heads are at tile positions lane*W + (set bits of hb)
            A acc = P::zero(), pre = P::zero();
            if (!__any_sync(FULL, c > 1)) {
                // at most one head per lane: it splits the run into the part
                // before it (pre) and the segment it opens (acc); selects only
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    const bool h = (hb >> i) & 1u;
                    pre = h ? acc : pre;
                    acc = h ? ((i == 0 && lane == 0) ? cin : P::zero()) : acc;
                    acc = P::fma(vs[lane * W + i], xv[i], acc);
                }
            } else {
                // general case: a head closes the open segment (the part
                // before the lane's first head belongs to an earlier segment)
                int cur = idx0 - 1;
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    if ((hb >> i) & 1u) {
                        // the closed segment opened at the lane's previous head
                        if (cur >= idx0)
                            emit(cur, acc,
                                 resolve ? lane * W + 31 - __clz(hb & ((1u << i) - 1u)) : 0);
                        else pre = acc;
                        ++cur;
                        acc = (i == 0 && lane == 0) ? cin : P::zero();
                    }
                    acc = P::fma(vs[lane * W + i], xv[i], acc);
                }
            }
            if (c == 0) pre = acc;  // the lane's total when it has no head
            const A v = acc;        // suffix if the lane has a head, else total
            const bool has = c > 0;

            // ---- cross-lane segmented sum of the open segments:
            // C_l = sum of v over lanes first_l..l, first_l = last lane <= l
            // with a head.  Short chains are summed serially, long ones by a
            // scan.
            const unsigned hm = __ballot_sync(FULL, has);
            const unsigned le = hm & ((lane == 31) ? FULL : ((2u << lane) - 1u));
            const int first = 31 - __clz(le);
            const int span = (int)__reduce_max_sync(FULL, (unsigned)(lane - first));
            A C = v;
            if (span <= 4) {
                for (int d = 1; d <= span; ++d) {
                    const A o = P::shfl_up(v, d);
                    if (lane - d >= first) C = P::add(C, o);
                }
            } else {
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const A o = P::shfl_up(C, d);
                    if (lane - d >= first) C = P::add(C, o);
                }
            }
            const A Cprev = P::shfl_up(C, 1);
            int prevpos = -1, openpos = -1;
            if (resolve) {  // head positions of the segments left open
                const int lastpos = c ? lane * W + 31 - __clz(hb) : -1;
                const unsigned below = hm & ((1u << lane) - 1u);
                prevpos = __shfl_sync(FULL, lastpos, below ? 31 - __clz(below) : 0);
                openpos = __shfl_sync(FULL, lastpos, first);
            }
            // a lane with a head closes the segment left open before it
            if (has && lane > 0) emit(idx0 - 1, P::add(Cprev, pre), prevpos);
            // the tile's last segment: stored, or carried if row `stop` goes on
            if (lane == 31) {
                *slot_carry = C;
                if (nseg == 1 && start == rF) {
                    *slot_f = C;  // still the bunch's first segment
                } else if (cont) {
                    if (t == t1 - 1) {  // continues into the next bunch
                        G = C;
                        hasG = true;
                    }  // else the next tile of this bunch stores it
                } else {
                    emit(nseg - 1, C, openpos);
                }
            }
            if (lane == 0) {
                a.tile_info[t] = (uint32_t)nseg | (dirty ? kInfoDirty : 0u) |
                                 (resolve ? kInfoResolved : 0u);
                if (dirty && !resolve) {  // kernel (c) re-arranges it
                    const uint32_t pos = atomicAdd(a.dirty_count, 1u);
                    if (pos < (uint32_t)ntiles) a.dirty_list[pos] = t;
                    else atomicOr(a.err, SSSPMV_DEV_CALIB);
                }
            }
            __syncwarp();
            carry = *slot_carry;
            ++q_con;
            issue_next();  // the stage just consumed takes the next copy
            start = start_nx;
            stop = stop_nx;
            pr_chunk = pr_nx;
            pr_chunk2 = pr_nx2;
        }
        // ---- synchronizer record of the bunch; its sums are finished in FP64
        __syncwarp();
        const A F = *slot_f;
        if (lane == 31) {
            a.sync_idx[cur] = rF;
            static_cast<double *>(a.sync_val)[cur] = P::to_f64(F);
            static_cast<double *>(a.tail_val)[cur] = hasG ? P::to_f64(G) : 0.0;
            a.tail_flag[cur] = hasG ? 1 : 0;
        }
        claim_next();
        cur = nxt;
        nxt = -1;
        if (cur >= nb) break;
        if constexpr (BATCHED) {
            if (ni != ci) {
                ci = ni;
                load_matrix(ci);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// kernel (c): calibration.  Block roles by blockIdx.x (the grid is one wave):
//   [0, nblk_sync)                  synchronizer sums, a warp per 32 bunches
//   [nblk_sync, +nblk_zero)         grid-stride zeroing of leading empty rows
//   [..., +nblk_tiles)              re-arrangement of the listed dirty tiles

struct CalibArgs {
    const int32_t *row_ptr;
    const int32_t *tile_offset;
    const uint32_t *tile_info;
    const int32_t *sync_idx;
    const void *sync_val;
    const void *tail_val;
    const int32_t *tail_flag;
    void *y;
    uint32_t *err;
    int32_t m;
    int32_t nnz;
    int32_t L;
    int64_t ntiles;
    int64_t nbunches;
    const uint32_t *dirty_count;  // written by kernel (b)
    const int32_t *dirty_list;
    int32_t nblk_tiles;
    int32_t nblk_sync;
    int32_t nblk_zero;
    uint32_t *spread_reset = nullptr;  // kernel (b)'s schedule flag, cleared here
    double alpha = 1.0, beta = 0.0;  // y = alpha A x + beta y (see SegsumArgs)
    int32_t axpby = 0;
    // batches only (see SegsumArgs)
    const BatchMat *mats = nullptr;
    const int32_t *bunch_mat = nullptr;
    const int32_t *totals = nullptr;
    int32_t count = 0;
};

constexpr int kCalibWarps = 8;

// the partials of dirty tile t (index in its matrix, rows [start, stop]) that
// belong to rows strictly inside (start, stop): one per non-empty row there,
// i.e. the tile's segments but the first and, when the tile's last row goes
// on into the next tile, the last.  rstop = row_ptr[stop] (any value when
// stop == m).  -1 when the count is impossible (0 <= K <= L).
__device__ __forceinline__ int32_t inner_partials(int32_t m, int32_t nnz, int32_t L, int64_t t,
                                                  int32_t stop, int32_t rstop, uint32_t info)
{
    const int32_t nseg = (int32_t)(info & kInfoSegMask);
    const int64_t e = (t + 1) * (int64_t)L < nnz ? (t + 1) * (int64_t)L : nnz;
    const bool cont = stop < m && (int64_t)rstop < e;
    const int32_t K = nseg - 1 - (cont ? 1 : 0);
    return (K < 0 || K > L) ? -1 : K;
}

// re-arrangement of one dirty tile by a warp (Sec. 3.2, checking
// prediction): the s-th partial (s >= 1, speculatively at y[start+s]) moves to
// the s-th non-empty row inside (start, stop), and the empty rows there become
// 0.  The partials are first read into registers (up to 64) or copied to the
// warp's shared buffer `part` (K <= L), so the rows can then be written in any
// order: the warp walks them forwards, eight chunks of 32 rows per round trip
// of row pointers.  The partials are read with the first chunk of row
// pointers and row_ptr[stop], so a tile over up to 256 rows costs one round
// trip of loads.
// t is the tile's index in its matrix, [start, stop] its rows.
template <class P>
__device__ __forceinline__ void repair_dirty_tile(const int32_t *__restrict__ row_ptr,
                                                  typename P::y_t *__restrict__ y, int32_t m,
                                                  int32_t nnz, int32_t L, int64_t t, int32_t start,
                                                  int32_t stop, uint32_t info, uint32_t *err,
                                                  int lane, typename P::y_t *part)
{
    using Y = typename P::y_t;
    const int32_t nseg = (int32_t)(info & kInfoSegMask);
    const int64_t e = (t + 1) * (int64_t)L < nnz ? (t + 1) * (int64_t)L : nnz;
    auto rp = [&](int32_t r) { return __ldg(row_ptr + (r < m ? r : m)); };
    constexpr int CH = 8;
    const int32_t rstop = rp(stop);
    // only the chunks that hold rows of (start, stop) or row_ptr[stop]
    int32_t pr[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
        pr[u] = start + 1 + 32 * u <= stop ? rp(start + 1 + 32 * u + lane) : 0;
    int32_t tail = (lane == 31 && start + 1 + 32 * CH <= stop) ? rp(start + 1 + 32 * CH) : 0;
    // K <= nseg - 1 partials (at most L, inside y): up to 64 stay in
    // registers, partial q at lane (q-1) % 32 of p0 (q <= 32) or p1; more go
    // to the warp's shared buffer
    int32_t qmax = nseg - 1 < L ? nseg - 1 : L;
    if (qmax > m - 1 - start) qmax = m - 1 - start;
    const bool inreg = qmax <= 64;
    Y p0 = Y(0), p1 = Y(0);
    if (inreg) {
        if (1 + lane <= qmax) p0 = y[start + 1 + lane];
        if (33 + lane <= qmax) p1 = y[start + 33 + lane];
    } else {
        for (int32_t q = 1 + lane; q <= qmax; q += 32) cp_async_g2s(part + q, y + start + q);
        cp_async_wait_all();
    }
    // the tile's last row goes on into the next tile: its segment is not
    // among the partials; non-empty rows strictly inside (start, stop) each
    // hold one segment
    const bool cont = stop < m && (int64_t)rstop < e;
    const int32_t K = nseg - 1 - (cont ? 1 : 0);
    if (K < 0 || K > L) {
        if (lane == 0) atomicOr(err, SSSPMV_DEV_CALIB);
        __syncwarp();
        return;
    }
    __syncwarp();
    int32_t before = 0;  // non-empty rows in (start, r) so far
    for (int32_t rb = start + 1; rb < stop; rb += 32 * CH) {
        if (rb != start + 1) {
#pragma unroll
            for (int u = 0; u < CH; ++u) pr[u] = rb + 32 * u <= stop ? rp(rb + 32 * u + lane) : 0;
            tail = (lane == 31 && rb + 32 * CH <= stop) ? rp(rb + 32 * CH) : 0;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            if (rb + 32 * u >= stop) break;  // no rows of the tile left
            const int32_t r = rb + 32 * u + lane;
            const int32_t lead = __shfl_sync(FULL, pr[u < CH - 1 ? u + 1 : CH - 1], 0);
            int32_t nx = __shfl_down_sync(FULL, pr[u], 1);
            if (lane == 31) nx = (u < CH - 1) ? lead : tail;
            const bool valid = r < stop;
            const bool ne = valid && nx > pr[u];
            const unsigned mask = __ballot_sync(FULL, ne);
            const int32_t q = before + 1 + __popc(mask & ((1u << lane) - 1u));
            Y pq = Y(0);
            if (inreg) {
                const Y a0 = __shfl_sync(FULL, p0, (q - 1) & 31);
                const Y a1 = __shfl_sync(FULL, p1, (q - 1) & 31);
                pq = q <= 32 ? a0 : a1;
            }
            if (valid) {
                Y v = Y(0);
                if (ne) {
                    if (q <= K) v = inreg ? pq : part[q];
                    else atomicOr(err, SSSPMV_DEV_CALIB);
                }
                y[r] = v;
            }
            before += __popc(mask);
        }
    }
    if (lane == 0 && before != K) atomicOr(err, SSSPMV_DEV_CALIB);
    __syncwarp();  // the buffer is reused for the warp's next tile
}


// the same re-arrangement by all kCalibWarps warps of a block, for a tile
// over many rows with K inner partials (inner_partials, checked by the
// caller): each warp takes a contiguous share of (start, stop) and
// counts its non-empty rows, keeping their flags as bit masks in `bits`
// (first pass, the only one that loads row pointers); after a block barrier
// it moves the partials from its count prefix on (second pass: stores
// only).  A tile over more than 32 * bits_words rows walks the row pointers
// again in the second pass.  Every thread of the block calls it with the
// same arguments; part holds L+1 values, cnt kCalibWarps.
template <class P>
__device__ void repair_long_tile(const int32_t *__restrict__ row_ptr,
                                 typename P::y_t *__restrict__ y, int32_t m,
                                 int32_t start, int32_t stop, int32_t K, uint32_t *err,
                                 typename P::y_t *part, int32_t *cnt, uint32_t *bits,
                                 int32_t bits_words, int32_t *stage, int32_t stage_chunks)
{
    using Y = typename P::y_t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int32_t q = 1 + (int32_t)threadIdx.x; q <= K; q += (int32_t)blockDim.x)
        cp_async_g2s(part + q, y + start + q);  // waited for after the count pass
    // this warp's rows [r0, r1) of (start, stop), shares a multiple of 32
    const int32_t n = stop - start - 1;
    const int32_t per = ((n + kCalibWarps - 1) / kCalibWarps + 31) & ~31;
    const int32_t r0 = start + 1 + warp * per;
    const int32_t r1 = r0 + per < stop ? r0 + per : stop;
    const bool keep = (n + 31) / 32 <= bits_words;
    // walks [r0, r1): f(first row of the chunk, r, valid, non-empty) per row,
    // chunk by chunk.  The row pointers of stage_chunks chunks (and the one
    // after them) are copied at a time into the warp's staging buffer by
    // asynchronous copies, so many are in flight without holding registers.
    int32_t *st = stage + warp * (32 * stage_chunks + 4);
    auto walk = [&](auto &&f) {
        for (int32_t rb = r0; rb < r1; rb += 32 * stage_chunks) {
            const int32_t nr = r1 - rb < 32 * stage_chunks ? r1 - rb : 32 * stage_chunks;
            for (int32_t i = lane; i <= nr; i += 32)
                cp_async_g2s(st + i, row_ptr + (rb + i < m ? rb + i : m));
            cp_async_wait_all();
            __syncwarp();
            for (int32_t c = 0; c < nr; c += 32) {
                const int32_t i = c + lane;
                const bool valid = i < nr;
                f(rb + c, rb + i, valid, valid && st[i + 1] > st[i]);
            }
            __syncwarp();  // the buffer is refilled next
        }
    };
    int32_t mine = 0;
    walk([&](int32_t rc, int32_t, bool, bool ne) {
        const unsigned mask = __ballot_sync(FULL, ne);
        mine += __popc(mask);
        if (keep && lane == 0 && rc < r1) bits[(rc - (start + 1)) >> 5] = mask;
    });
    cp_async_wait_all();
    if (lane == 0) cnt[warp] = mine;
    __syncthreads();  // counts, flags and partials in place
    int32_t before = 0, total = 0;
    for (int w = 0; w < kCalibWarps; ++w) {
        const int32_t c = cnt[w];
        if (w < warp) before += c;
        total += c;
    }
    if (threadIdx.x == 0 && total != K) atomicOr(err, SSSPMV_DEV_CALIB);
    // row r (valid: inside this warp's share) from its chunk's flags
    auto place = [&](int32_t r, bool valid, unsigned mask) {
        const bool ne = (mask >> lane) & 1u;
        const int32_t q = before + 1 + __popc(mask & ((1u << lane) - 1u));
        if (valid) {
            Y v = Y(0);
            if (ne) {
                if (q <= K) v = part[q];
                else atomicOr(err, SSSPMV_DEV_CALIB);
            }
            y[r] = v;
        }
        before += __popc(mask);
    };
    if (keep) {
        for (int32_t rc = r0; rc < r1; rc += 32)
            place(rc + lane, rc + lane < r1, bits[(rc - (start + 1)) >> 5]);
    } else {
        walk([&](int32_t, int32_t r, bool valid, bool ne) {
            place(r, valid, __ballot_sync(FULL, ne));
        });
    }
    __syncthreads();  // part, cnt and bits are reused by the block's next tile
}

// the batch matrix holding global tile t: the last one whose first tile is
// at or before t (matrices without tiles share the next one's base)
__device__ __forceinline__ int32_t batch_matrix_of_tile(const BatchMat *mats, int32_t count,
                                                        int64_t t)
{
    int32_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if ((int64_t)__ldg(&mats[mid].tile_base) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class P, bool BATCHED = false>
__global__ void __launch_bounds__(kCalibWarps * 32) calibrate_kernel(const CalibArgs a)
{
    using Y = typename P::y_t;
    using A = typename P::acc_t;
    grid_dep_wait();  // everything below reads kernel (b)'s results
    if (a.spread_reset != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.spread_reset = 0u;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    extern __shared__ __align__(16) unsigned char calib_smem[];
    Y *part = reinterpret_cast<Y *>(calib_smem) + (size_t)warp * (a.L + 1);  // tile role only
    Y *__restrict__ y = static_cast<Y *>(a.y);
    const int64_t ntiles = BATCHED ? (int64_t)__ldg(a.totals) : a.ntiles;
    const int64_t nbunches = BATCHED ? (int64_t)__ldg(a.totals + 1) : a.nbunches;
    // ---- re-arrangement of dirty tiles (Sec. 3.2, checking prediction).
    // Kernel (b) appended every dirty tile it left speculative to a list
    // (the paper's speculator, in any order).  The tile role's warps stride
    // over the list, consecutive entries going to consecutive blocks, and read
    // up to 32 of their entries and tile flags in one round of loads.  A tile
    // over more than kLongRepairRows rows is re-arranged by a whole block: for
    // a single matrix, by the synchronizer and zeroing blocks once their own
    // work is done (block b takes the long tiles among t = b (mod their
    // count), found from the tile offsets, so that the long tiles at the
    // sparse end of a matrix go to consecutive blocks); in a batch, by the
    // tile-role block whose warp meets it in the list.
    // a block's long tiles: index, rows [start, stop], inner partials
    __shared__ int32_t s_long[kLongListCap], s_lst[kLongListCap], s_lsp[kLongListCap],
        s_lK[kLongListCap];
    __shared__ int32_t s_nlong, s_cnt[kCalibWarps];
    int64_t count = (int64_t)*(volatile const uint32_t *)a.dirty_count;
    if (count > ntiles) count = ntiles;  // kernel (b) appends each tile at most once
    // the matrix data of global tile t (in a batch: of its matrix)
    struct Tile {
        const int32_t *row_ptr;
        Y *y;
        int32_t m, nnz, start, stop;
        int64_t t;  // in its matrix
    };
    auto tile_of = [&](int64_t t) -> Tile {
        if constexpr (BATCHED) {
            const int32_t mi = batch_matrix_of_tile(a.mats, a.count, t);
            const BatchMat *mm = a.mats + mi;
            const int32_t tb = __ldg(&mm->tile_base);
            const int32_t *to = a.tile_offset + tb + mi;  // the matrix's offsets
            return Tile{ldg_ptr(&mm->row_ptr),
                        static_cast<Y *>(ldg_ptr(const_cast<void *const *>(&mm->y))),
                        __ldg(&mm->m), __ldg(&mm->nnz), __ldg(to + (t - tb)),
                        __ldg(to + (t - tb) + 1), t - tb};
        } else {
            return Tile{a.row_ptr, y, a.m, a.nnz, __ldg(a.tile_offset + t),
                        __ldg(a.tile_offset + t + 1), t};
        }
    };
    // an entry must name a dirty tile that kernel (b) did not resolve
    auto listed_ok = [&](int64_t t, uint32_t info) {
        return t >= 0 && t < ntiles && (info & kInfoDirty) && !(info & kInfoResolved);
    };
    // the block's long tiles, kept in s_long: the first warp's buffer takes
    // the partials; the other warps' buffers stage row pointers (up to 16
    // chunks of 32 per warp and pass, leaving at least 1,024 words) and hold
    // the non-empty flags
    Y *bpart = reinterpret_cast<Y *>(calib_smem);
    uint32_t *bits = reinterpret_cast<uint32_t *>(bpart + (a.L + 1));
    const int32_t rest_words =
        (int32_t)((size_t)(kCalibWarps - 1) * (size_t)(a.L + 1) * sizeof(Y) / 4);
    int32_t stage_chunks = ((rest_words - 1024) / kCalibWarps - 4) / 32;
    if (stage_chunks > 16) stage_chunks = 16;
    const int32_t stage_words = kCalibWarps * (32 * stage_chunks + 4);
    const int32_t bits_words = rest_words - stage_words;
    int32_t *stage = reinterpret_cast<int32_t *>(bits + bits_words);
    auto repair_kept = [&]() {
        __syncthreads();  // s_long complete
        const int nl = s_nlong < kLongListCap ? s_nlong : kLongListCap;
        for (int i = 0; i < nl; ++i) {
            Tile T;
            if constexpr (BATCHED) T = tile_of(s_long[i]);  // the matrix's arrays
            else T = Tile{a.row_ptr, y, a.m, a.nnz, s_lst[i], s_lsp[i], s_long[i]};
            if (s_lK[i] >= 0)  // the same for every thread of the block
                repair_long_tile<P>(T.row_ptr, T.y, T.m, s_lst[i], s_lsp[i], s_lK[i], a.err,
                                    bpart, s_cnt, bits, bits_words, stage, stage_chunks);
        }
        __syncthreads();
    };
    // (single matrix) the long dirty tiles among t = b0 (mod nb), in rounds
    // of kLongListCap tiles, kLongListCap / 256 per thread with their loads
    // in flight together (a round cannot overflow s_long)
    auto repair_long_strided = [&](int64_t b0, int64_t nb) {
        constexpr int U = kLongListCap / (kCalibWarps * 32);
        const int64_t per_round = (int64_t)kLongListCap * nb;
        for (int64_t base = b0; base < ntiles; base += per_round) {
            if (threadIdx.x == 0) s_nlong = 0;
            __syncthreads();
            int32_t st[U], sp[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t t = base + (int64_t)(threadIdx.x + u * kCalibWarps * 32) * nb;
                st[u] = t < ntiles ? __ldg(a.tile_offset + t) : 0;
                sp[u] = t < ntiles ? __ldg(a.tile_offset + t + 1) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t t = base + (int64_t)(threadIdx.x + u * kCalibWarps * 32) * nb;
                if (t < ntiles && sp[u] - st[u] > kLongRepairRows) {
                    // the flags and row_ptr[stop] in one round
                    const uint32_t info = __ldg(a.tile_info + t);
                    const int32_t rstop = __ldg(a.row_ptr + (sp[u] < a.m ? sp[u] : a.m));
                    if (listed_ok(t, info)) {
                        const int32_t K = inner_partials(a.m, a.nnz, a.L, t, sp[u], rstop, info);
                        if (K < 0) {
                            atomicOr(a.err, SSSPMV_DEV_CALIB);
                        } else {
                            const int slot = atomicAdd(&s_nlong, 1);
                            s_long[slot] = (int32_t)t;
                            s_lst[slot] = st[u];
                            s_lsp[slot] = sp[u];
                            s_lK[slot] = K;
                        }
                    }
                }
            }
            repair_kept();
        }
    };
    int blk = blockIdx.x;
    if (blk < a.nblk_sync + a.nblk_zero) {
        if (blk < a.nblk_sync) {
            // ---- synchronization (Alg. 1's synchronization step, on the GPU):
            // the run of bunches sharing a first row adds into that row, plus the
            // tail partial the bunch before the run left for it.  A warp covers
            // 32 bunches, one per lane; runs are summed by a segmented warp scan
            // and a run that goes on past the window is finished by this warp.
            const double *sv = static_cast<const double *>(a.sync_val);
            const double *tv = static_cast<const double *>(a.tail_val);
            // (in a batch, runs are keyed by matrix and row: bunches of different
            // matrices never share a row)
            auto key_of = [&](int64_t ww) -> int64_t {
                const int64_t r = __ldg(a.sync_idx + ww);
                if constexpr (BATCHED) return ((int64_t)__ldg(a.bunch_mat + ww) << 32) | r;
                else return r;
            };
            // windows of 32 bunches, one per warp, strided over the role's warps
            for (int64_t wi = (int64_t)blk * kCalibWarps + warp; wi * 32 < nbunches;
                 wi += (int64_t)a.nblk_sync * kCalibWarps) {
                const int64_t base = wi * 32;
                const int64_t w = base + lane;
                const bool valid = w < nbunches;
                const int64_t kw = valid ? key_of(w) : -1;
                const int32_t r = (int32_t)(kw & 0xffffffff);
                int64_t kprev = __shfl_up_sync(FULL, kw, 1);
                if (lane == 0) kprev = (valid && w > 0) ? key_of(w - 1) : -1;
                const bool lead = valid && (w == 0 || kprev != kw);
                Y *__restrict__ yw = y;  // y and m of this lane's bunch's matrix
                int32_t mw = a.m;
                if constexpr (BATCHED) {
                    if (valid) {
                        const BatchMat *mm = a.mats + (kw >> 32);
                        yw = static_cast<Y *>(ldg_ptr(const_cast<void *const *>(&mm->y)));
                        mw = __ldg(&mm->m);
                    }
                }
                // this bunch's partial and the tail partial the bunch before it left
                // (used if this lane leads its run), loaded in the same round as the
                // keys
                double C = valid ? sv[w] : 0.0;
                // (lane 31) the next window's first key, in the same round
                const int64_t knext =
                    (lane == 31 && valid && w + 1 < nbunches) ? key_of(w + 1) : -2;
                double tprev = 0.0;
                if (valid && w > 0) {
                    const int32_t f = __ldg(a.tail_flag + w - 1);
                    const double v = tv[w - 1];  // read unconditionally, kept only if flagged
                    tprev = f ? v : 0.0;
                }
                const unsigned lmask = __ballot_sync(FULL, lead);
                if (lmask == 0) continue;  // the whole window continues a run led earlier
                const int firstlead = __ffs(lmask) - 1;
                const bool owned = valid && lane >= firstlead;
                // segmented inclusive sum over runs (heads: leaders and invalid lanes)
                const bool head = lead || !valid;
                const unsigned hmask = __ballot_sync(FULL, head) | 1u;
                const unsigned le = hmask & ((lane == 31) ? FULL : ((2u << lane) - 1u));
                const int first = 31 - __clz(le);
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const double o = __shfl_up_sync(FULL, C, d);
                    if (lane - d >= first) C += o;
                }
                // does this lane's run go on to the next bunch?
                bool next_same;
                const bool next_lead = __shfl_down_sync(FULL, lead, 1);
                const bool next_valid = __shfl_down_sync(FULL, valid, 1);
                if (lane < 31) next_same = next_valid && !next_lead;
                else next_same = valid && w + 1 < nbunches && knext == kw;
                const double tlead = __shfl_sync(FULL, tprev, first);  // of the run's leader
                if (owned && !next_same) {
                    const double total = C + tlead;
                    if (r >= 0 && r < mw) yw[r] = scaled_store_value(yw, r, (Y)total, a.alpha, a.beta, a.axpby);
                    else atomicOr(a.err, SSSPMV_DEV_RANGE);
                }
                const bool open = __shfl_sync(FULL, owned && next_same, 31);
                if (open) {  // the last run continues past the window (long rows)
                    const int64_t kk = __shfl_sync(FULL, kw, 31);
                    const int32_t rr = (int32_t)(kk & 0xffffffff);
                    const double csum = __shfl_sync(FULL, C, 31);
                    const double ctail = __shfl_sync(FULL, tlead, 31);
                    // eight windows of 32 bunches per round trip of loads (a row of
                    // 10^6 entries spans hundreds of bunches); each lane still adds
                    // its bunches in increasing order, so the sum does not change
                    constexpr int U = 8;
                    double acc = 0.0;
                    for (int64_t b2 = base + 32;; b2 += 32 * U) {
                        bool in[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int64_t ww = b2 + 32 * u + lane;
                            in[u] = ww < nbunches && key_of(ww) == kk;
                        }
                        bool full = true;
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (in[u]) acc += sv[b2 + 32 * u + lane];
                            full = full && __all_sync(FULL, in[u]);
                        }
                        if (!full) break;
                    }
#pragma unroll
                    for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(FULL, acc, d);
                    Y *__restrict__ yr =
                        reinterpret_cast<Y *>(__shfl_sync(FULL, (unsigned long long)yw, 31));
                    const int32_t mr = __shfl_sync(FULL, mw, 31);
                    if (lane == 0) {
                        const double total = csum + acc + ctail;
                        if (rr >= 0 && rr < mr)
                            yr[rr] = scaled_store_value(yr, rr, (Y)total, a.alpha, a.beta, a.axpby);
                        else atomicOr(a.err, SSSPMV_DEV_RANGE);
                    }
                }
            }
        } else {
            blk -= a.nblk_sync;
            // ---- rows before tile_offset[0] are empty and covered by no tile (in
            // a batch: each matrix's, the role's warps striding over the matrices)
            if constexpr (BATCHED) {
                for (int32_t mi = blk * kCalibWarps + warp; mi < a.count;
                     mi += a.nblk_zero * kCalibWarps) {  // a warp per matrix
                    const BatchMat *mm = a.mats + mi;
                    const int32_t r0 = __ldg(a.tile_offset + __ldg(&mm->tile_base) + mi);
                    Y *__restrict__ ym = static_cast<Y *>(ldg_ptr(const_cast<void *const *>(&mm->y)));
                    for (int32_t r = lane; r < r0; r += 32)
                        ym[r] = scaled_store_value(ym, r, Y(0), a.alpha, a.beta, a.axpby);
                }
            } else {
                const int32_t r0 = __ldg(a.tile_offset);
                for (int64_t r = (int64_t)blk * blockDim.x + threadIdx.x; r < r0;
                     r += (int64_t)a.nblk_zero * blockDim.x)
                    y[r] = scaled_store_value(y, r, Y(0), a.alpha, a.beta, a.axpby);
            }
        }
        // these blocks are done long before the tile role's warps
        if constexpr (!BATCHED) {
            if (count > 0) repair_long_strided(blockIdx.x, (int64_t)a.nblk_sync + a.nblk_zero);
        }
        return;
    }
    blk -= a.nblk_sync + a.nblk_zero;
    const int64_t nw = (int64_t)a.nblk_tiles * kCalibWarps;
    if constexpr (BATCHED) {
        if (threadIdx.x == 0) s_nlong = 0;
        __syncthreads();
    }
    // the other dirty tiles, a warp each (in a batch, long ones are kept for
    // the block while there is room)
    for (int64_t i0 = (int64_t)warp * a.nblk_tiles + blk; i0 < count; i0 += nw * 32) {
        const int64_t il = i0 + (int64_t)lane * nw;
        const int64_t tl = il < count ? (int64_t)__ldg(a.dirty_list + il) : -1;
        const bool okt = tl >= 0 && tl < ntiles;
        const uint32_t infl = okt ? __ldg(a.tile_info + tl) : 0u;
        // (single matrix) the window's tile offsets in the same round
        int32_t st_l = 0, sp_l = 0;
        if (!BATCHED && okt) {
            st_l = __ldg(a.tile_offset + tl);
            sp_l = __ldg(a.tile_offset + tl + 1);
        }
        const bool good = listed_ok(tl, infl);
        if (il < count && !good) atomicOr(a.err, SSSPMV_DEV_CALIB);
        // (single matrix) long tiles were taken by the scan above
        unsigned todo = __ballot_sync(FULL, good && (BATCHED || sp_l - st_l <= kLongRepairRows));
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t t = __shfl_sync(FULL, tl, src);
            const uint32_t info = __shfl_sync(FULL, infl, src);
            Tile T;
            if constexpr (BATCHED) {
                T = tile_of(t);
                if (T.stop - T.start > kLongRepairRows) {
                    int slot = 0;
                    if (lane == 0) slot = atomicAdd(&s_nlong, 1);
                    slot = __shfl_sync(FULL, slot, 0);
                    if (slot < kLongListCap) {
                        const int32_t rstop = __ldg(T.row_ptr + (T.stop < T.m ? T.stop : T.m));
                        const int32_t K = inner_partials(T.m, T.nnz, a.L, T.t, T.stop, rstop, info);
                        if (lane == 0) {
                            s_long[slot] = (int32_t)t;
                            s_lst[slot] = T.start;
                            s_lsp[slot] = T.stop;
                            s_lK[slot] = K;
                            if (K < 0) atomicOr(a.err, SSSPMV_DEV_CALIB);
                        }
                        continue;
                    }
                }
            } else {
                T = Tile{a.row_ptr, y, a.m, a.nnz, __shfl_sync(FULL, st_l, src),
                         __shfl_sync(FULL, sp_l, src), t};
            }
            repair_dirty_tile<P>(T.row_ptr, T.y, T.m, T.nnz, a.L, T.t, T.start, T.stop, info,
                                 a.err, lane, part);
        }
    }
    if constexpr (BATCHED) repair_kept();
}

}  // namespace ssspmv
