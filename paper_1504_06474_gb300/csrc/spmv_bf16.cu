// spmv_bf16.cu -- BF16-value instantiations: val in bfloat16, x and y in float,
// compensated FP32 accumulation as in spmv_f32.cu.
#include "launch.cuh"

namespace ssspmv {

int bf16_supported_w(int32_t *out, int cap)
{
    int n = 0;
#define X(w) if (n < cap) out[n] = w; ++n;
    SSSPMV_SHAPES(X)
#undef X
    return n;
}

int bf16_resolve(Layout &l, int32_t S_opt)
{
    switch (l.W) {
#define X(w) case w: resolve_bunches<BF16C, w>(l, S_opt); return SSSPMV_OK;
        SSSPMV_SHAPES(X)
#undef X
    default: return SSSPMV_EUNSUPPORTED;
    }
}

int bf16_run(Call &c)
{
    switch (c.lay.W) {
#define X(w) case w: return run_shape<BF16C, w>(c);
        SSSPMV_SHAPES(X)
#undef X
    default: return SSSPMV_EUNSUPPORTED;
    }
}

}  // namespace ssspmv
