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

struct Layout {
    int32_t W = 0, L = 0, S = 0;
    int64_t ntiles = 0, nbunches = 0, nbunch_cap = 0;
    size_t off_tile_offset = 0, off_tile_info = 0, off_sync_idx = 0, off_sync_val = 0,
           off_tail_val = 0, off_tail_flag = 0, off_err = 0, total = 0;
};

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

inline void carve(Layout &l)
{
    size_t o = 0;
    l.off_err = o;
    o = align256(o + 16);
    l.off_tile_offset = o;
    o = align256(o + sizeof(int32_t) * (size_t)(l.ntiles + 1));
    l.off_tile_info = o;
    o = align256(o + sizeof(uint32_t) * (size_t)(l.ntiles > 0 ? l.ntiles : 1));
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

}  // namespace ssspmv
