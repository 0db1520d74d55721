// layout.h -- tile shape resolution and workspace carve-up (host side).
#pragma once
#include <cstddef>
#include <cstdint>

#include "ssspmv.h"

// odd W values (entries per lane) compiled for every precision
#define SSSPMV_SHAPES(X) X(15) X(21) X(27) X(31)

namespace ssspmv {

// tiles per thread-bunch when the caller does not choose S: small bunches,
// handed out dynamically, balance tiles that differ in cost (many empty rows)
constexpr int32_t kDefaultS = 4;

// the automatic S of a single product: kDefaultS, but fewer for matrices of
// under 98,304 tiles, so that each of the ~3,000 resident warps of a large GPU
// still gets about ten bunches and the ticket pool can balance them (and the
// spread schedule has shares to split); the same on every device, so the
// workspace size does not depend on it
inline int32_t auto_bunch_tiles(int64_t ntiles)
{
    const int64_t s = (ntiles + 32767) / 32768;
    return (int32_t)(s < 1 ? 1 : (s > kDefaultS ? kDefaultS : s));
}

// The four words at the front of a workspace (uint32 each):
//   [0] device error bits          cleared by kernel (a)
//   [1] bunch ticket of kernel (b) cleared by kernel (a)
//   [2] dirty-tile count           cleared by kernel (a); kernel (b) appends
//                                  the dirty tiles it leaves to kernel (c)
//   [3] kernel (b)'s schedule flag set by kernel (a) when it sees runs of
//                                  empty rows, cleared by kernel (c)
// (a plan execution, which skips kernel (a), clears words 0..2 and keeps the
// plan's flag)
constexpr int kWordErr = 0, kWordTicket = 1, kWordDirty = 2, kWordSpread = 3;
constexpr size_t kHeaderBytes = 16;

struct Layout {
    int32_t W = 0, L = 0, S = 0;
    int64_t ntiles = 0, nbunches = 0, nbunch_cap = 0;
    size_t off_tile_offset = 0, off_tile_info = 0, off_dirty_list = 0, off_sync_idx = 0,
           off_sync_val = 0, off_tail_val = 0, off_tail_flag = 0, off_err = 0, total = 0;
};

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

inline void carve(Layout &l)
{
    size_t o = 0;
    l.off_err = o;
    o = align256(o + kHeaderBytes);
    l.off_tile_offset = o;
    o = align256(o + sizeof(int32_t) * (size_t)(l.ntiles + 1));
    l.off_tile_info = o;
    o = align256(o + sizeof(uint32_t) * (size_t)(l.ntiles > 0 ? l.ntiles : 1));
    // the dirty tiles kernel (b) leaves to kernel (c), in any order
    l.off_dirty_list = o;
    o = align256(o + sizeof(int32_t) * (size_t)(l.ntiles > 0 ? l.ntiles : 1));
    const size_t nb = (size_t)(l.nbunch_cap > 0 ? l.nbunch_cap : 1);
    l.off_sync_idx = o;
    o = align256(o + sizeof(int32_t) * nb);
    l.off_sync_val = o;
    o = align256(o + sizeof(double) * nb);
    l.off_tail_val = o;
    o = align256(o + sizeof(double) * nb);
    l.off_tail_flag = o;
    o = align256(o + sizeof(int32_t) * nb);
    l.total = o;
}

// workspace carve-up of a batch (one 64-byte record per matrix, BatchMat)
constexpr size_t kBatchMatBytes = 64;

struct BatchLayout {
    int32_t W = 0, L = 0, S = 0;
    int64_t cap_tiles = 0, cap_bunches = 0;
    size_t off_err = 0, off_mats = 0, off_toff = 0, off_info = 0, off_dirty = 0, off_bmat = 0,
           off_sidx = 0, off_sval = 0, off_tval = 0, off_tflag = 0, total = 0;
};

// the words at the front of a batch workspace: error bits, bunch ticket,
// totals {tiles, bunches} (written by the set-up kernel), dirty-tile count
constexpr int kBatchWordDirty = 4;

inline void batch_layout(int32_t count, int64_t total_nnz, int32_t W, int32_t S, BatchLayout &l)
{
    l.W = W;
    l.L = 32 * W;
    l.S = S;
    l.cap_tiles = (total_nnz + l.L - 1) / l.L + count;
    l.cap_bunches = (l.cap_tiles + S - 1) / S + count;
    size_t o = 0;
    l.off_err = o;  // err word, ticket, totals {tiles, bunches}, dirty-tile count
    o = align256(o + 32);
    l.off_mats = o;
    o = align256(o + kBatchMatBytes * (size_t)(count > 0 ? count : 1));
    l.off_toff = o;
    o = align256(o + sizeof(int32_t) * (size_t)(l.cap_tiles + count));
    l.off_info = o;
    o = align256(o + sizeof(uint32_t) * (size_t)(l.cap_tiles > 0 ? l.cap_tiles : 1));
    l.off_dirty = o;
    o = align256(o + sizeof(int32_t) * (size_t)(l.cap_tiles > 0 ? l.cap_tiles : 1));
    const size_t nb = (size_t)(l.cap_bunches > 0 ? l.cap_bunches : 1);
    l.off_bmat = o;
    o = align256(o + sizeof(int32_t) * nb);
    l.off_sidx = o;
    o = align256(o + sizeof(int32_t) * nb);
    l.off_sval = o;
    o = align256(o + sizeof(double) * nb);
    l.off_tval = o;
    o = align256(o + sizeof(double) * nb);
    l.off_tflag = o;
    o = align256(o + sizeof(int32_t) * nb);
    l.total = o;
}

}  // namespace ssspmv
