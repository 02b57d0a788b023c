// Throughput probes of the arithmetic units the hot path's kernels lean on,
// measured on the device the library runs on (the roofline's ALU peaks):
// FP64 FMA, FP32 FMA and the MUFU base-2 exponential.  Each kernel runs
// eight independent dependency chains per thread over a grid of four
// 256-thread blocks per SM, long enough (tens of ms) that launch overhead is
// negligible; the host times it with CUDA events.
#include <cuda_runtime.h>

#include "../../include/pimd.h"

namespace {

constexpr int PROBE_ITERS = 4096;

__global__ void __launch_bounds__(256) probe_fma64(double a, double b, double* sink)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = a + 0.001 * (threadIdx.x + k);
    for (int i = 0; i < PROBE_ITERS; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], b, a);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 1.2345) sink[0] = s;  // never true: keeps the chains alive
}

__global__ void __launch_bounds__(256) probe_fma32(float a, float b, float* sink)
{
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = a + 0.001f * (threadIdx.x + k);
    for (int i = 0; i < 4 * PROBE_ITERS; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __fmaf_rn(x[k], b, a);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 1.2345f) sink[0] = s;
}

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 0.25 - 2^x stays in [-0.75, 0.25) for x in [-1, 1); one ex2 and one FP32
// add per step, eight independent chains per thread.
__global__ void __launch_bounds__(256) probe_ex2(float a, float* sink)
{
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = -a * (float)(threadIdx.x + 37 * k + 1) * 1e-3f;
    for (int i = 0; i < PROBE_ITERS; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __fadd_rn(0.25f, -ex2f(x[k]));
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s = __fmaf_rn(s, 1.0001f, x[k]);
    if (s == 1.2345f) sink[0] = s;
}

template <class F>
double time_ms(cudaStream_t st, F&& launch, cudaError_t* err)
{
    cudaEvent_t a, b;
    *err = cudaEventCreate(&a);
    if (*err != cudaSuccess) return 0.0;
    *err = cudaEventCreate(&b);
    if (*err != cudaSuccess) {
        cudaEventDestroy(a);
        return 0.0;
    }
    launch();  // warm-up
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    *err = cudaEventSynchronize(b);
    float ms = 0.f;
    if (*err == cudaSuccess) *err = cudaEventElapsedTime(&ms, a, b);
    if (*err == cudaSuccess) *err = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

extern "C" pimd_status pimd_probe_rates(double* sink, pimd_rates* out, void* stream)
{
    if (!sink || !out) return PIMD_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PIMD_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = 4 * sms, threads = 256;
    const double lanes = (double)grid * threads * 8;
    cudaError_t e;
    const double t64 = time_ms(st, [&] { probe_fma64<<<grid, threads, 0, st>>>(1.0, 0.999, sink); }, &e);
    if (e != cudaSuccess) return PIMD_ECUDA;
    const double t32 = time_ms(st, [&] { probe_fma32<<<grid, threads, 0, st>>>(1.0f, 0.999f, (float*)sink); }, &e);
    if (e != cudaSuccess) return PIMD_ECUDA;
    const double tx = time_ms(st, [&] { probe_ex2<<<grid, threads, 0, st>>>(1.0f, (float*)sink); }, &e);
    if (e != cudaSuccess) return PIMD_ECUDA;
    out->fp64_tflops = 2.0 * lanes * PROBE_ITERS / (t64 * 1e-3) / 1e12;
    out->fp32_tflops = 2.0 * lanes * 4 * PROBE_ITERS / (t32 * 1e-3) / 1e12;
    out->ex2_per_s = lanes * PROBE_ITERS / (tx * 1e-3);
    out->sms = sms;
    return PIMD_OK;
}

cudaError_t xdf_launch_probe_chain(const double* Q, const double* G, const double* y0, const double* s, int nblk,
                                   int n_iter, int split, double* y_out, long long* cycles, cudaStream_t st);

extern "C" pimd_status pimd_probe_chain(int nblk, int n_iter, int split, const double* Q, const double* G,
                                        const double* y0, const double* s, double* y_out, long long* cycles,
                                        void* stream)
{
    if (!Q || !G || !y0 || !s || !y_out || !cycles) return PIMD_EINVAL;
    if (nblk < 1 || nblk > 8 || n_iter < 1 || (split != 1 && split != 2 && split != 4)) return PIMD_EINVAL;
    const cudaError_t e = xdf_launch_probe_chain(Q, G, y0, s, nblk, n_iter, split, y_out, cycles,
                                                 (cudaStream_t)stream);
    return e == cudaSuccess ? PIMD_OK : PIMD_ECUDA;
}
