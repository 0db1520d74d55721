// spmv_f64.cu -- FP64 instantiations (val, x, y and accumulation in double).
#include "launch.cuh"

namespace ssspmv {

int f64_supported_w(int32_t *out, int cap)
{
    int n = 0;
#define X(w) if (n < cap) out[n] = w; ++n;
    SSSPMV_SHAPES(X)
#undef X
    return n;
}

int f64_resolve(Layout &l, int32_t S_opt)
{
    switch (l.W) {
#define X(w) case w: resolve_bunches<F64, w>(l, S_opt); return SSSPMV_OK;
        SSSPMV_SHAPES(X)
#undef X
    default: return SSSPMV_EUNSUPPORTED;
    }
}

int f64_run(Call &c)
{
    switch (c.lay.W) {
#define X(w) case w: return run_shape<F64, w>(c);
        SSSPMV_SHAPES(X)
#undef X
    default: return SSSPMV_EUNSUPPORTED;
    }
}

}  // namespace ssspmv
