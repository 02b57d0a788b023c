// Device-side building blocks shared by the sm_103a kernels of the PIMD hot path.
//
// Wide-exponent floats ("Wef"): the exchange recursions (arXiv 2404.02628,
// Sec. III) multiply factors exp(+-kappa |dr|^2) whose logarithms reach
// thousands, far outside FP64's exponent range, while every sum they enter has
// only non-negative terms.  A Wef keeps an FP64 mantissa in [1,2) (or 0) and a
// separate 32-bit binary exponent, so products are exact to FP64 rounding and
// sums never overflow or underflow; no logarithm or exponential is taken on the
// dependent chain of the recursion.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <mutex>

#define PIMD_TB 32            // exchange tile edge: 32 rows x 32 columns, one warp lane per row
#define WEF_ZERO_E (-(1 << 29))
#define WEF_SAT_E (1 << 28)

struct Wef {
    double m;
    int e;
};

// 2^k as a double for k in [-1022, 1023]; 0 below.  Built from the bit pattern.
__device__ __forceinline__ double pow2i(int k)
{
    return (k < -1022) ? 0.0 : __hiloint2double((k + 1023) << 20, 0);
}

// m * 2^k for m in [1,2) (or 0) and k <= 0: integer add into the exponent field.
__device__ __forceinline__ double scale_down(double m, int k)
{
    if (k < -1022 || m == 0.0) return 0.0;
    return __hiloint2double(__double2hiint(m) + (k << 20), __double2loint(m));
}

__device__ __forceinline__ Wef wef_zero() { return Wef{0.0, WEF_ZERO_E}; }

// Normalise a non-negative finite mantissa (normal or zero) into [1,2).
__device__ __forceinline__ Wef wef_norm(double m, int e)
{
    if (!(m > 0.0)) {
        if (m == 0.0) return wef_zero();
        return Wef{m, e};  // NaN propagates
    }
    int hi = __double2hiint(m);
    int ex = ((hi >> 20) & 0x7FF) - 1023;
    hi = (hi & 0x800FFFFF) | 0x3FF00000;
    int en = e + ex;
    if (en < WEF_ZERO_E / 2) return wef_zero();
    return Wef{__hiloint2double(hi, __double2loint(m)), en};
}

__device__ __forceinline__ Wef wef_mul(Wef a, Wef b) { return wef_norm(a.m * b.m, a.e + b.e); }

__device__ __forceinline__ Wef wef_add(Wef a, Wef b)
{
    if (a.e >= b.e) return wef_norm(a.m + scale_down(b.m, b.e - a.e), a.e);
    return wef_norm(b.m + scale_down(a.m, a.e - b.e), b.e);
}

// Cody-Waite split of ln 2: LN2_HI carries 33 significant bits so n*LN2_HI is
// exact for |n| < 2^20; LN2_LO = ln 2 - LN2_HI rounded to FP64.
#define PIMD_LN2_HI __longlong_as_double(0x3fe62e42fef00000LL)
#define PIMD_LN2_LO 7.440617110012397e-11
#define PIMD_LOG2E 1.4426950408889634

// e^x as a Wef for any x (x = -inf gives zero; overflowing exponents give NaN).
__device__ __forceinline__ Wef wef_exp(double x)
{
    if (x == -INFINITY) return wef_zero();
    double t = floor(x * PIMD_LOG2E);
    if (t < (double)(WEF_ZERO_E / 2)) return wef_zero();
    if (!(t < (double)WEF_SAT_E)) return Wef{__longlong_as_double(0x7ff8000000000000LL), 0};
    double r = fma(-t, PIMD_LN2_HI, x);
    r = fma(-t, PIMD_LN2_LO, r);
    return wef_norm(exp(r), (int)t);
}

// ln of a Wef (zero gives -inf).
__device__ __forceinline__ double wef_log(Wef a)
{
    if (a.m == 0.0) return -INFINITY;
    return log(a.m) + fma((double)a.e, PIMD_LN2_HI, (double)a.e * PIMD_LN2_LO);
}

// Plain double value of a Wef (underflows to 0, overflows to inf).
__device__ __forceinline__ double wef_to_double(Wef a)
{
    if (a.m == 0.0) return 0.0;
    if (a.e > 1023) return INFINITY;
    if (a.e >= -1022) return a.m * pow2i(a.e);
    if (a.e < -1100) return 0.0;
    return (a.m * pow2i(a.e + 64)) * pow2i(-64);
}

// ---------------------------------------------------------------------------
// Bounded cross-block waits.  A waiter polls with acquire loads; after
// spin_limit polls, or as soon as another block has raised the shared error
// word, it records the failure and returns false, so no kernel ever hangs.

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

enum { PIMD_DEVERR_TIMEOUT = 1, PIMD_DEVERR_RANGE = 2 };

__device__ __forceinline__ bool wait_flag(const int* flag, int want, int* err, int spin_limit, int code_site)
{
    for (int it = 0; it < spin_limit; ++it) {
        if (ld_acquire(flag) >= want) return true;
        if ((it & 63) == 63 && ld_acquire(err) != 0) return false;
        __nanosleep(it < 64 ? 0 : 64);
    }
    atomicCAS(err, 0, (PIMD_DEVERR_TIMEOUT << 24) | (code_site & 0xFFFFFF));
    return false;
}

// Block-wide barrier for code where lanes of a warp may have taken different
// paths just before (e.g. lane-0-only stores or waits): bar.sync is
// warp-aligned, so the warp is reconverged first.
__device__ __forceinline__ void block_sync()
{
    __syncwarp();
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of NV doubles (blockDim.x a multiple of 32,
// at most 1024).  Result valid in thread 0.

template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* smem /* 32*NV */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    block_sync();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) smem[w * NV + q] = v[q];
    block_sync();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int i = 0; i < nw; ++i) s += smem[i * NV + q];
            v[q] = s;
        }
    }
    block_sync();
}

// ---------------------------------------------------------------------------
// Host side: one-time set-up per device (kernel attributes such as the
// dynamic shared-memory opt-in belong to the device that is current when they
// are set).  set() runs under a lock, with the device current, until it
// succeeds once on that device.

struct DeviceOnce {
    std::mutex mu;
    bool done[128] = {};
};

template <class F>
inline cudaError_t device_once(DeviceOnce& o, F&& set)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(o.mu);
    if (o.done[dev]) return cudaSuccess;
    e = set();
    if (e == cudaSuccess) o.done[dev] = true;
    return e;
}

// Poll count of the bounded device waits when a call's configuration leaves
// it at 0: the PIMD_SPIN_LIMIT environment variable if set to a positive
// integer (lets tests drive the timeout paths of calls that take no
// configuration), otherwise 2^24.
inline int default_spin_limit(int configured)
{
    if (configured > 0) return configured;
    const char* s = getenv("PIMD_SPIN_LIMIT");
    if (s && *s) {
        const long v = strtol(s, nullptr, 10);
        if (v > 0 && v < (1L << 30)) return (int)v;
    }
    return 1 << 24;
}
