// probe.cu -- throughput probes that measure the denominators of the ALU
// rooflines on the device at hand: the FP32 fused multiply-add rate and the
// special-function (base-2 exponential) rate.  No counterpart in the paper;
// the blend kernels are bound by these two units rather than by HBM.
#include "gsr_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent dependency chains per thread
constexpr int PROBE_UNROLL = 32;  // rounds per loop trip (loop overhead < 2 %)

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(float *out, int iters, float x, float y)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; it += PROBE_UNROLL) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    out[(int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float v)
{
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_exp(float *out, int iters)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; it += PROBE_UNROLL) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = ex2_approx(-a[k]);  // stays in (0, 1]
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    out[(int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

// y = __expf(x): the exponential the blend kernels evaluate alpha with, for a
// test that checks its error against the bound the parity margins assume
__global__ void k_probe_expf(const float *__restrict__ x, float *__restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __expf(x[i]);
}

gsr_status probe_args(float *out, int32_t blocks, int32_t iters)
{
    if (!out || blocks <= 0 || iters <= 0 || iters % PROBE_UNROLL) return GSR_ERR_INVALID_ARG;
    return GSR_OK;
}

} // namespace

extern "C" {

GSR_API gsr_status gsr_probe_fma(float *out, int32_t blocks, int32_t iters, void *stream)
{
    const gsr_status st = probe_args(out, blocks, iters);
    if (st != GSR_OK) return st;
    k_probe_fma<<<(unsigned)blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(out, iters, 0.9999999f, 1e-7f);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

GSR_API gsr_status gsr_probe_exp(float *out, int32_t blocks, int32_t iters, void *stream)
{
    const gsr_status st = probe_args(out, blocks, iters);
    if (st != GSR_OK) return st;
    k_probe_exp<<<(unsigned)blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(out, iters);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

GSR_API gsr_status gsr_probe_expf(const float *x, float *y, int64_t n, void *stream)
{
    if (!x || !y || n <= 0) return GSR_ERR_INVALID_ARG;
    k_probe_expf<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

} // extern "C"
