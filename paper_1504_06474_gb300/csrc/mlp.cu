// mlp.cu -- the learned variant selector's device code: the row_ptr feature
// kernel and the FP32 forward, backward and Adam kernels of a small
// multilayer perceptron (ReLU hidden layers, linear outputs, squared loss).
// Not in the paper: the selector only picks among the library's kernels and
// never changes their arithmetic.
#include <cuda_runtime.h>

#include <cmath>

#include "launch.cuh"

namespace ssspmv {

// ---------------------------------------------------------------------------
// features: one pass over the row lengths, block partial sums into 64-bit
// global counters, then one thread turns the counters into the 16 features

constexpr int kFeatThreads = 256;
constexpr int kHistBins = 32;  // bin b: row length in [2^(b-1), 2^b), bin 0: empty

// counter layout (unsigned long long)
enum {
    FC_SUM2 = 0,        // sum of len^2
    FC_MAX,             // max len
    FC_EMPTY,           // empty rows
    FC_SHORT,           // rows with len <= 4
    FC_HEAVY,           // rows with len >= 2 * mean (needs the mean: second pass)
    FC_LONGNNZ,         // entries in rows longer than 1024
    FC_JUMP,            // rows whose length differs from the previous row's by more than 2x
    FC_EMPTYRUN,        // empty rows followed by an empty row
    FC_XNNZ,            // entries in rows of at least 32 * mean (second pass)
    FC_HIST,            // kHistBins counters
    FC_COUNT = FC_HIST + kHistBins
};

__device__ __forceinline__ int len_bin(int32_t len)
{
    return len <= 0 ? 0 : (32 - __clz((unsigned)len) < kHistBins ? 32 - __clz((unsigned)len)
                                                                  : kHistBins - 1);
}

// pass 1 (second == 0) or pass 2 (second == 1, the mean known)
__global__ void __launch_bounds__(kFeatThreads)
    feature_count_kernel(const int32_t *__restrict__ row_ptr, int32_t m, int32_t nnz, int second,
                         unsigned long long *__restrict__ cnt)
{
    __shared__ unsigned long long s[FC_COUNT];
    for (int i = threadIdx.x; i < FC_COUNT; i += blockDim.x) s[i] = 0ull;
    __syncthreads();
    const double mean = m > 0 ? (double)nnz / (double)m : 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long sum2 = 0, mx = 0, empty = 0, shrt = 0, heavy = 0, longnnz = 0, jump = 0,
                       erun = 0, xnnz = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride) {
        const int32_t a = __ldg(row_ptr + r), b = __ldg(row_ptr + r + 1);
        const int32_t len = b - a;
        if (!second) {
            sum2 += (unsigned long long)len * (unsigned long long)len;
            mx = len > (int64_t)mx ? (unsigned long long)len : mx;
            empty += len == 0;
            shrt += len <= 4;
            if (len > 1024) longnnz += (unsigned long long)len;
            if (r > 0) {
                const int32_t p = a - __ldg(row_ptr + r - 1);
                jump += (len > 2 * p + 1) || (p > 2 * len + 1);
                erun += (len == 0) && (p == 0);
            }
            atomicAdd(&s[FC_HIST + len_bin(len)], 1ull);
        } else {
            heavy += (double)len >= 2.0 * mean;
            if ((double)len >= 32.0 * mean) xnnz += (unsigned long long)len;
        }
    }
    atomicAdd(&s[FC_SUM2], sum2);
    atomicMax(&s[FC_MAX], mx);
    atomicAdd(&s[FC_EMPTY], empty);
    atomicAdd(&s[FC_SHORT], shrt);
    atomicAdd(&s[FC_HEAVY], heavy);
    atomicAdd(&s[FC_LONGNNZ], longnnz);
    atomicAdd(&s[FC_JUMP], jump);
    atomicAdd(&s[FC_EMPTYRUN], erun);
    atomicAdd(&s[FC_XNNZ], xnnz);
    __syncthreads();
    for (int i = threadIdx.x; i < FC_COUNT; i += blockDim.x) {
        if (i == FC_MAX) atomicMax(cnt + i, s[i]);
        else if (s[i]) atomicAdd(cnt + i, s[i]);
    }
}

// the 16 features, each of order one
__global__ void feature_finish_kernel(const unsigned long long *__restrict__ cnt, int32_t m,
                                      int32_t n, int32_t nnz, float *__restrict__ f)
{
    if (threadIdx.x != 0) return;
    const double md = m > 0 ? (double)m : 1.0;
    const double mean = (double)nnz / md;
    const double var = (double)cnt[FC_SUM2] / md - mean * mean;
    const double sd = var > 0 ? sqrt(var) : 0.0;
    const double nz = nnz > 0 ? (double)nnz : 1.0;
    // histogram percentiles as log2 lengths
    double q[3] = {0.5, 0.9, 0.99}, pv[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (int b = 0; b < kHistBins; ++b) {
            acc += (double)cnt[FC_HIST + b];
            if (acc >= q[k] * md) {
                pv[k] = (double)b;
                break;
            }
        }
    }
    f[0] = (float)(log2(md + 1.0) / 24.0);
    f[1] = (float)(log2((double)nnz + 1.0) / 32.0);
    f[2] = (float)(log2(mean + 1.0) / 8.0);
    f[3] = (float)(sd / (mean + 1.0));
    f[4] = (float)(log2((double)cnt[FC_MAX] + 1.0) / 24.0);
    f[5] = (float)((double)cnt[FC_EMPTY] / md);
    f[6] = (float)((double)cnt[FC_SHORT] / md);
    f[7] = (float)((double)cnt[FC_HEAVY] / md);
    f[8] = (float)((double)cnt[FC_LONGNNZ] / nz);
    f[9] = (float)(pv[0] / 16.0);
    f[10] = (float)(pv[1] / 16.0);
    f[11] = (float)(pv[2] / 16.0);
    f[12] = (float)((double)cnt[FC_JUMP] / md);
    f[13] = (float)(log2(480.0 / (mean + 1e-9) + 1.0) / 16.0);  // rows per 480-entry tile
    f[14] = (float)((double)cnt[FC_EMPTYRUN] / md);
    f[15] = (float)((double)cnt[FC_XNNZ] / nz);
    (void)n;
}

int run_features(const int32_t *row_ptr, int32_t m, int32_t n, int32_t nnz, float *out,
                 void *scratch, cudaStream_t s)
{
    unsigned long long *cnt = static_cast<unsigned long long *>(scratch);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * FC_COUNT, s);
    if (e != cudaSuccess) return record_cuda_error(e);
    int64_t blocks = ((int64_t)m + kFeatThreads - 1) / kFeatThreads;
    const int64_t cap = 8LL * device_sm_count();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    for (int pass = 0; pass < 2; ++pass)
        feature_count_kernel<<<(unsigned)blocks, kFeatThreads, 0, s>>>(row_ptr, m, nnz, pass, cnt);
    feature_finish_kernel<<<1, 32, 0, s>>>(cnt, m, n, nnz, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_error(e);
    return SSSPMV_OK;
}

size_t features_scratch_bytes() { return sizeof(unsigned long long) * FC_COUNT; }

// ---------------------------------------------------------------------------
// dense layers of the perceptron, FP32.  Weights row-major W[O][I].

constexpr int kMlpThreads = 256;

// out[b][o] = act(sum_i W[o][i] * in[b][i] + bias[o]); pre[b][o] keeps the
// pre-activation for the backward pass (may be null)
__global__ void __launch_bounds__(kMlpThreads)
    dense_forward_kernel(const float *__restrict__ in, const float *__restrict__ Wt,
                         const float *__restrict__ bias, float *__restrict__ pre,
                         float *__restrict__ out, int B, int I, int O, int relu)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)B * O) return;
    const int b = (int)(k / O), o = (int)(k % O);
    float acc = bias[o];
    for (int i = 0; i < I; ++i) acc = fmaf(Wt[o * I + i], in[(int64_t)b * I + i], acc);
    if (pre) pre[k] = acc;
    out[k] = relu ? fmaxf(acc, 0.0f) : acc;
}

// squared loss over the outputs whose target is finite (mask: target NaN =
// not measured): g = 2 (out - target) / count, loss accumulated in *loss
__global__ void __launch_bounds__(kMlpThreads)
    loss_grad_kernel(const float *__restrict__ out, const float *__restrict__ target,
                     float *__restrict__ g, int64_t n, float inv_count, float *loss)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (k < n) {
        const float t = target[k];
        const float d = (t == t) ? out[k] - t : 0.0f;
        g[k] = 2.0f * d * inv_count;
        l = d * d * inv_count;
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) l += __shfl_xor_sync(FULL, l, s);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

// dW[o][i] = sum_b g[b][o] * in[b][i];  db[o] = sum_b g[b][o]  (one thread
// per weight, a fixed order over the batch: deterministic)
__global__ void __launch_bounds__(kMlpThreads)
    dense_grad_w_kernel(const float *__restrict__ in, const float *__restrict__ g,
                        float *__restrict__ dW, float *__restrict__ db, int B, int I, int O)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < (int64_t)O * I) {
        const int o = (int)(k / I), i = (int)(k % I);
        float acc = 0.0f;
        for (int b = 0; b < B; ++b) acc = fmaf(g[(int64_t)b * O + o], in[(int64_t)b * I + i], acc);
        dW[k] = acc;
    } else if (k < (int64_t)O * I + O) {
        const int o = (int)(k - (int64_t)O * I);
        float acc = 0.0f;
        for (int b = 0; b < B; ++b) acc += g[(int64_t)b * O + o];
        db[o] = acc;
    }
}

// gin[b][i] = (sum_o W[o][i] * g[b][o]) * (pre_in[b][i] > 0)  (ReLU below)
__global__ void __launch_bounds__(kMlpThreads)
    dense_grad_in_kernel(const float *__restrict__ Wt, const float *__restrict__ g,
                         const float *__restrict__ pre_in, float *__restrict__ gin, int B, int I,
                         int O)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)B * I) return;
    const int b = (int)(k / I), i = (int)(k % I);
    float acc = 0.0f;
    for (int o = 0; o < O; ++o) acc = fmaf(Wt[o * I + i], g[(int64_t)b * O + o], acc);
    gin[k] = pre_in[k] > 0.0f ? acc : 0.0f;
}

// Adam (Kingma & Ba 2015) on n parameters, step t >= 1
__global__ void __launch_bounds__(kMlpThreads)
    adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                float *__restrict__ m2, int64_t n, float lr, float b1, float b2, float eps,
                float wd, int t)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k] + wd * p[k];
    const float a = b1 * m1[k] + (1.0f - b1) * gk;
    const float v = b2 * m2[k] + (1.0f - b2) * gk * gk;
    m1[k] = a;
    m2[k] = v;
    const float ah = a / (1.0f - powf(b1, (float)t));
    const float vh = v / (1.0f - powf(b2, (float)t));
    p[k] -= lr * ah / (sqrtf(vh) + eps);
}

// argmin over each row of the predictions (the chosen class)
__global__ void argmin_kernel(const float *__restrict__ out, int B, int K, int32_t *__restrict__ cls)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    int best = 0;
    float bv = out[(int64_t)b * K];
    for (int k = 1; k < K; ++k) {
        const float v = out[(int64_t)b * K + k];
        if (v < bv) {
            bv = v;
            best = k;
        }
    }
    cls[b] = best;
}

static unsigned blocks_for(int64_t n) { return (unsigned)((n + kMlpThreads - 1) / kMlpThreads); }

}  // namespace ssspmv

using namespace ssspmv;

// parameter block layout: W1[H1][F] b1[H1] W2[H2][H1] b2[H2] W3[K][H2] b3[K]
static int64_t mlp_param_count(int F, int H1, int H2, int K)
{
    return (int64_t)H1 * F + H1 + (int64_t)H2 * H1 + H2 + (int64_t)K * H2 + K;
}

extern "C" {

size_t ssspmv_features_scratch_bytes(void) { return features_scratch_bytes(); }

int ssspmv_features(int32_t m, int32_t n, int32_t nnz, const int32_t *row_ptr, float *features,
                    void *scratch, void *stream)
{
    if (m < 0 || n < 0 || nnz < 0 || (m > 0 && !row_ptr) || !features || !scratch)
        return SSSPMV_EINVAL;
    return run_features(row_ptr, m, n, nnz, features, scratch, static_cast<cudaStream_t>(stream));
}

int64_t ssspmv_mlp_param_count(int32_t F, int32_t H1, int32_t H2, int32_t K)
{
    if (F <= 0 || H1 <= 0 || H2 <= 0 || K <= 0) return 0;
    return mlp_param_count(F, H1, H2, K);
}

size_t ssspmv_mlp_scratch_floats(int32_t B, int32_t F, int32_t H1, int32_t H2, int32_t K)
{
    // pre1, act1, pre2, act2 (B x H), out (B x K), gout (B x K), g2 (B x H2), g1 (B x H1), loss
    return (size_t)B * (2 * H1 + 2 * H2 + 2 * K + H2 + H1) + 1;
}

static int mlp_forward_impl(const float *params, const float *X, int32_t B, int32_t F, int32_t H1,
                            int32_t H2, int32_t K, float *scratch, cudaStream_t s)
{
    const float *W1 = params, *b1 = W1 + (int64_t)H1 * F;
    const float *W2 = b1 + H1, *b2 = W2 + (int64_t)H2 * H1;
    const float *W3 = b2 + H2, *b3 = W3 + (int64_t)K * H2;
    float *pre1 = scratch, *act1 = pre1 + (int64_t)B * H1;
    float *pre2 = act1 + (int64_t)B * H1, *act2 = pre2 + (int64_t)B * H2;
    float *out = act2 + (int64_t)B * H2;
    dense_forward_kernel<<<blocks_for((int64_t)B * H1), kMlpThreads, 0, s>>>(X, W1, b1, pre1, act1,
                                                                            B, F, H1, 1);
    dense_forward_kernel<<<blocks_for((int64_t)B * H2), kMlpThreads, 0, s>>>(act1, W2, b2, pre2,
                                                                            act2, B, H1, H2, 1);
    dense_forward_kernel<<<blocks_for((int64_t)B * K), kMlpThreads, 0, s>>>(act2, W3, b3, nullptr,
                                                                           out, B, H2, K, 0);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SSSPMV_OK : record_cuda_error(e);
}

int ssspmv_mlp_forward(const float *params, const float *X, int32_t B, int32_t F, int32_t H1,
                       int32_t H2, int32_t K, float *scratch, float *out, void *stream)
{
    if (!params || !X || !scratch || B <= 0 || F <= 0 || H1 <= 0 || H2 <= 0 || K <= 0)
        return SSSPMV_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = mlp_forward_impl(params, X, B, F, H1, H2, K, scratch, s);
    if (rc) return rc;
    if (out) {
        const float *o = scratch + (int64_t)B * (2 * H1 + 2 * H2);
        cudaError_t e = cudaMemcpyAsync(out, o, sizeof(float) * (size_t)B * K,
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    return SSSPMV_OK;
}

int ssspmv_mlp_backward(const float *params, const float *X, const float *target, int32_t B,
                        int32_t F, int32_t H1, int32_t H2, int32_t K, float *scratch, float *grad,
                        float *loss, void *stream)
{
    if (!params || !X || !target || !scratch || !grad || B <= 0 || F <= 0 || H1 <= 0 ||
        H2 <= 0 || K <= 0)
        return SSSPMV_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = mlp_forward_impl(params, X, B, F, H1, H2, K, scratch, s);
    if (rc) return rc;
    const float *W2 = params + (int64_t)H1 * F + H1;
    const float *W3 = W2 + (int64_t)H2 * H1 + H2;
    float *pre1 = scratch, *act1 = pre1 + (int64_t)B * H1;
    float *pre2 = act1 + (int64_t)B * H1, *act2 = pre2 + (int64_t)B * H2;
    float *out = act2 + (int64_t)B * H2, *gout = out + (int64_t)B * K;
    float *g2 = gout + (int64_t)B * K, *g1 = g2 + (int64_t)B * H2;
    float *lacc = g1 + (int64_t)B * H1;
    float *dW1 = grad, *db1 = dW1 + (int64_t)H1 * F;
    float *dW2 = db1 + H1, *db2 = dW2 + (int64_t)H2 * H1;
    float *dW3 = db2 + H2, *db3 = dW3 + (int64_t)K * H2;
    cudaError_t e = cudaMemsetAsync(lacc, 0, sizeof(float), s);
    if (e != cudaSuccess) return record_cuda_error(e);
    // squared error averaged over all B*K outputs; a NaN target (a class not
    // measured) contributes neither loss nor gradient
    const int64_t n = (int64_t)B * K;
    loss_grad_kernel<<<blocks_for(n), kMlpThreads, 0, s>>>(out, target, gout, n, 1.0f / (float)n,
                                                          lacc);
    dense_grad_w_kernel<<<blocks_for((int64_t)K * H2 + K), kMlpThreads, 0, s>>>(act2, gout, dW3,
                                                                              db3, B, H2, K);
    dense_grad_in_kernel<<<blocks_for((int64_t)B * H2), kMlpThreads, 0, s>>>(W3, gout, pre2, g2, B,
                                                                            H2, K);
    dense_grad_w_kernel<<<blocks_for((int64_t)H2 * H1 + H2), kMlpThreads, 0, s>>>(act1, g2, dW2,
                                                                                db2, B, H1, H2);
    dense_grad_in_kernel<<<blocks_for((int64_t)B * H1), kMlpThreads, 0, s>>>(W2, g2, pre1, g1, B,
                                                                            H1, H2);
    dense_grad_w_kernel<<<blocks_for((int64_t)H1 * F + H1), kMlpThreads, 0, s>>>(X, g1, dW1, db1,
                                                                               B, F, H1);
    if (loss) {
        e = cudaMemcpyAsync(loss, lacc, sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? SSSPMV_OK : record_cuda_error(e);
}

int ssspmv_mlp_adam(float *params, const float *grad, float *m1, float *m2, int64_t n, float lr,
                    float beta1, float beta2, float eps, float weight_decay, int32_t step,
                    void *stream)
{
    if (!params || !grad || !m1 || !m2 || n <= 0 || step < 1) return SSSPMV_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    adam_kernel<<<blocks_for(n), kMlpThreads, 0, s>>>(params, grad, m1, m2, n, lr, beta1, beta2,
                                                     eps, weight_decay, step);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SSSPMV_OK : record_cuda_error(e);
}

int ssspmv_mlp_select(const float *params, const float *X, int32_t B, int32_t F, int32_t H1,
                      int32_t H2, int32_t K, float *scratch, int32_t *cls, void *stream)
{
    if (!cls) return SSSPMV_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = ssspmv_mlp_forward(params, X, B, F, H1, H2, K, scratch, nullptr, stream);
    if (rc) return rc;
    const float *out = scratch + (int64_t)B * (2 * H1 + 2 * H2);
    argmin_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(out, B, K, cls);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SSSPMV_OK : record_cuda_error(e);
}

}  // extern "C"
