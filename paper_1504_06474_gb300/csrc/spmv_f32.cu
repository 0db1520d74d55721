// spmv_f32.cu -- FP32 instantiations: val, x, y in float; each segment sum is an
// unevaluated pair s + c updated by TwoProduct/TwoSum (compensated FP32).
#include "launch.cuh"

namespace ssspmv {

int f32_supported_w(int32_t *out, int cap)
{
    int n = 0;
#define X(w) if (n < cap) out[n] = w; ++n;
    SSSPMV_SHAPES(X)
#undef X
    return n;
}

int f32_resolve(Layout &l, int32_t S_opt)
{
    switch (l.W) {
#define X(w) case w: resolve_bunches<F32C, w>(l, S_opt); return SSSPMV_OK;
        SSSPMV_SHAPES(X)
#undef X
    default: return SSSPMV_EUNSUPPORTED;
    }
}

int f32_run(Call &c)
{
    switch (c.lay.W) {
#define X(w) case w: return run_shape<F32C, w>(c);
        SSSPMV_SHAPES(X)
#undef X
    default: return SSSPMV_EUNSUPPORTED;
    }
}

}  // namespace ssspmv
