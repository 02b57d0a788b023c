// Per-(slice, particle-block) units of the springs (a1) and the trap + pair
// forces (a4), shared by their own kernels and by the force workers of the
// persistent exchange launch.  Block coordinates and shared-memory scratch
// come in as arguments; blockDim.x threads, one particle per thread.
#pragma once
#include "pimd_md.cuh"

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// double -> float by truncating the significand (round toward zero) with
// integer operations: on GB300 the hardware F2F.F32.F64 conversion costs
// about twice an FP64 FMA, the bit manipulation a few integer-pipe ops.
// Relative error below 2^-23; values below the float normal range give a
// signed zero and values above it (and NaN) an infinity of the same sign.
__device__ __forceinline__ float d2f_trunc(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    const unsigned s = hi & 0x80000000u;
    unsigned b = s | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    b = e <= 0 ? s : b;
    b = e >= 255 ? (s | 0x7F800000u) : b;
    return __uint_as_float(b);
}

// float -> double on the integer pipe (exact), every case by bit
// manipulation so that no FP64-pipe conversion is ever issued (a predicated
// one would be, in every thread): the exponent rebiased and the significand
// shifted into place; zero keeps its sign, a subnormal is normalised with a
// leading-zero count, infinities and NaN keep an all-ones exponent.
__device__ __forceinline__ double f2d_exact(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned sgn = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    unsigned hi = sgn | ((e - 127u + 1023u) << 20) | (m >> 3), lo = m << 29;
    if (e == 0xFFu) hi = sgn | 0x7FF00000u | (m >> 3);
    if (e == 0u) {
        // m 2^-149: the highest set bit s of m becomes the implicit one
        const int s = 31 - __clz(m | 1u);
        const unsigned long long f = ((unsigned long long)(m ^ (1u << s))) << (52 - s);
        hi = m == 0u ? sgn : (sgn | ((unsigned)(s + 874) << 20) | (unsigned)(f >> 32));
        lo = m == 0u ? 0u : (unsigned)f;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// FP64 <-> double-float on the integer pipe: the FP64 conversions and adds
// run on the FP64 pipe, which on this part is the bottleneck of the
// thermostat kernels, so both directions take the bit fields apart instead.
// FP64 -> df: the high part is x with its significand truncated to 24 bits,
// the low part the remaining 29 significand bits as a float (rounded to 24
// bits: about 2^-47 relative overall).  Exponents outside [-70, 100] (and
// zero, infinities, NaN) take the FP64 route.
// The rare wide-range cases of d2df / df2d on the FP64 pipe, out of line so
// that the common path never issues them as predicated instructions.
static __device__ __noinline__ df d2df_wide(double x)
{
    const float h = d2f_trunc(x);
    return df{h, d2f_trunc(x - (double)h)};
}
static __device__ __noinline__ double df2d_wide(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df d2df(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int E = (int)((hi >> 20) & 0x7FFu) - 1023;
    if (E < -70 || E > 100) return d2df_wide(x);
    const unsigned sgn = hi & 0x80000000u;
    const float h = __uint_as_float(sgn | ((unsigned)(E + 127) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
    const float scale = __uint_as_float((unsigned)(E - 52 + 127) << 23);  // 2^(E-52), a normal float
    const float l = __uint_as_float(__float_as_uint(__uint2float_rn(lo & 0x1FFFFFFFu) * scale) | sgn);
    return df{h, l};
}

// df -> FP64: the 24-bit significand of h widened to 53 bits, the low part's
// significand added (or subtracted) at its offset, one renormalising shift.
// Bits of l below the FP64 unit are truncated (at most 2 ulp).  Parts outside
// the normal range, or an l too large for a normalised pair, take the FP64
// route.
__device__ __forceinline__ double df2d(df a)
{
    const unsigned hb = __float_as_uint(a.h), lb = __float_as_uint(a.l);
    const int Eh = (int)((hb >> 23) & 0xFFu) - 127;
    const int El = (int)((lb >> 23) & 0xFFu) - 127;
    const int sh = El - Eh + 29;  // offset of l's significand in units of 2^(Eh-52)
    const bool l_zero = (lb & 0x7FFFFFFFu) == 0u;
    if (Eh < -100 || Eh > 100 || (!l_zero && (El == -127 || sh > 6))) return df2d_wide(a);
    unsigned long long M = (unsigned long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;
    int E = Eh;
    if (!l_zero && sh > -25) {
        const unsigned long long ml = (lb & 0x7FFFFFu) | 0x800000u;
        const unsigned long long L = sh >= 0 ? ml << sh : ml >> (-sh);
        if ((hb ^ lb) & 0x80000000u) {
            M -= L;
            if (M < (1ull << 52)) {
                M <<= 1;
                E -= 1;
            }
        } else {
            M += L;
            if (M >= (1ull << 53)) {
                M >>= 1;
                E += 1;
            }
        }
    }
    const unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                    ((unsigned long long)(E + 1023) << 52) | (M & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}
// (a1) Internal ring-polymer springs (Sec. III interior-bead formula and the
// within-particle half of the exterior-bead formulas): F_l^j = -k (2 r^j -
// r^{j+1} - r^{j-1}), with the missing neighbour of beads 1 and P dropped.
// Also the slice's part of sum_l E_int^(l) (always FP64) into part[j*gx + bx].
__device__ __forceinline__ void springs_unit(const BeadView& b, const ForceParams& fp, double* f, double* part, int bx, int j,
                                             int gx, double* red /* [32] */)
{
    const int l = bx * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (l < b.N) {
        for (int c = 0; c < b.d; ++c) {
            const size_t o = ((size_t)j * b.d + c) * b.ld + l;
            const double x = b.r[o];
            const double xm = (j > 0) ? b.r[o - (size_t)b.d * b.ld] : x;
            const double xp = (j < b.P - 1) ? b.r[o + (size_t)b.d * b.ld] : x;
            double fo;
            if (fp.mixed) {
                const float xf = d2f_trunc(x);
                fo = (double)(-(float)fp.ks * ((xf - d2f_trunc(xm)) + (xf - d2f_trunc(xp))));
            } else {
                fo = -fp.ks * ((x - xm) + (x - xp));
            }
            f[o] = fp.accumulate ? f[o] + fo : fo;
            if (j < b.P - 1) e = fma(xp - x, xp - x, e);
        }
    }
    double v[1] = {0.5 * fp.ks * e};
    block_reduce<1>(v, red);
    if (threadIdx.x == 0) part[j * gx + bx] = v[0];
}

// (a4) Trap + Gaussian pairs in slice `by` for particles [bx*PT, bx*PT + PT)
// (Sec. II U, Sec. IV B): F += -grad(V_slice)/P; (energy, virial) partials
// into part[2*(by*gx + bx)].  FP64 arithmetic.
template <int D, int PT>
__device__ __forceinline__ void pair_unit_f64(const BeadView& b, const ForceParams& fp, double* f, double* part, int bx,
                                              int by, int gx, double* sx /* [D * PT] */, double* red /* [64] */)
{
    if (bx * PT >= b.N) {  // a block past this replica's particles
        if (threadIdx.x == 0) {
            part[2 * (by * gx + bx) + 0] = 0.0;
            part[2 * (by * gx + bx) + 1] = 0.0;
        }
        return;
    }
    const int i = bx * PT + threadIdx.x, j = by;
    const double* rs = b.r + (size_t)j * D * b.ld;
    double xi[D], g[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        xi[c] = (i < b.N) ? rs[(size_t)c * b.ld + i] : 0.0;
        g[c] = 0.0;
    }
    double esum = 0.0;
    if (fp.A != 0.0) {
        for (int k0 = 0; k0 < b.N; k0 += PT) {
            const int k = k0 + threadIdx.x;
#pragma unroll
            for (int c = 0; c < D; ++c) sx[c * PT + threadIdx.x] = (k < b.N) ? rs[(size_t)c * b.ld + k] : 0.0;
            __syncthreads();
            const int kn = min(PT, b.N - k0);
            for (int kk = 0; kk < kn; ++kk) {
                double q2 = 0.0, dx[D];
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    dx[c] = xi[c] - sx[c * PT + kk];
                    q2 = fma(dx[c], dx[c], q2);
                }
                double ee = (k0 + kk == i) ? 0.0 : exp(-q2 * fp.inv_s2);
                esum += ee;
#pragma unroll
                for (int c = 0; c < D; ++c) g[c] = fma(ee, dx[c], g[c]);
            }
            __syncthreads();
        }
    }
    double v[2] = {0.0, 0.0};
    if (i < b.N) {
        const double cpair = -2.0 * fp.A * fp.inv_s2;  // grad_i of A e^{-q2/s2} = cpair * e * dx
        double t2 = 0.0, vir = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double grad = fp.omega2 * xi[c] + cpair * g[c];
            const size_t o = ((size_t)j * D + c) * b.ld + i;
            const double fo = -grad * fp.inv_P;
            f[o] = fp.accumulate ? f[o] + fo : fo;
            t2 = fma(xi[c], xi[c], t2);
            vir = fma(xi[c], grad, vir);
        }
        v[0] = 0.5 * fp.omega2 * t2 + 0.5 * fp.A * esum;
        v[1] = vir;
    }
    block_reduce<2>(v, red);
    if (threadIdx.x == 0) {
        part[2 * (by * gx + bx) + 0] = v[0];
        part[2 * (by * gx + bx) + 1] = v[1];
    }
}

// FP32 pair arithmetic with exp2 on the MUFU unit; coordinates pre-scaled by
// sqrt(log2(e))/s so that each pair costs one ex2 and no extra multiply; one
// particle per thread, partners two at a time on the packed FP32x2 pipe.
template <int D, int PT>
__device__ __forceinline__ void pair_unit_f32(const BeadView& b, const ForceParams& fp, double* f, double* part, int bx,
                                              int by, int gx, float2* sx /* [D * PT / 2] */, double* red /* [64] */)
{
    if (bx * PT >= b.N) {  // a block past this replica's particles
        if (threadIdx.x == 0) {
            part[2 * (by * gx + bx) + 0] = 0.0;
            part[2 * (by * gx + bx) + 1] = 0.0;
        }
        return;
    }
    const int i = bx * PT + threadIdx.x, j = by;
    const double* rs = b.r + (size_t)j * D * b.ld;
    const float sc = fp.sc32;
    float xf[D];
    float2 xi[D], g[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        xf[c] = (i < b.N) ? d2f_trunc(rs[(size_t)c * b.ld + i]) : 0.f;
        const float xs = xf[c] * sc;
        xi[c] = make_float2(xs, xs);
        g[c] = make_float2(0.f, 0.f);
    }
    float2 esum = make_float2(0.f, 0.f);
    if (fp.A != 0.0) {
        for (int k0 = 0; k0 < b.N; k0 += PT) {
            const int k = k0 + threadIdx.x;
            float* sxf = reinterpret_cast<float*>(sx);
#pragma unroll
            for (int c = 0; c < D; ++c)
                sxf[c * PT + threadIdx.x] = (k < b.N) ? -d2f_trunc(rs[(size_t)c * b.ld + k]) * sc : -1.0e18f;
            __syncthreads();
            // partner pairs holding at least one particle (the padding past N
            // sits at -1e18 and adds exp2(-inf) = 0)
            const int nkk = (min(PT, b.N - k0) + 1) >> 1;
#pragma unroll 4
            for (int kk = 0; kk < nkk; ++kk) {
                float2 dx[D];
#pragma unroll
                for (int c = 0; c < D; ++c) dx[c] = __fadd2_rn(xi[c], sx[c * (PT / 2) + kk]);
                float2 q2 = __fmul2_rn(dx[0], dx[0]);
#pragma unroll
                for (int c = 1; c < D; ++c) q2 = __ffma2_rn(dx[c], dx[c], q2);
                const float2 ee = make_float2(ex2_approx(-q2.x), ex2_approx(-q2.y));
                esum = __fadd2_rn(esum, ee);
#pragma unroll
                for (int c = 0; c < D; ++c) g[c] = __ffma2_rn(ee, dx[c], g[c]);
            }
            __syncthreads();
        }
    }
    // per-particle epilogue in FP32 (mixed precision: the pair and trap
    // forces are FP32 quantities); the force is added to the FP64 array and
    // the block's energy and virial are summed in FP64
    double v[2] = {0.0, 0.0};
    if (i < b.N) {
        const float cpair = (float)fp.cpair32, om2 = (float)fp.omega2, mip = -(float)fp.inv_P;
        float t2 = 0.f, vir = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float grad = fmaf(om2, xf[c], cpair * (g[c].x + g[c].y));
            const size_t o = ((size_t)j * D + c) * b.ld + i;
            const double fo = f2d_exact(grad * mip);
            f[o] = fp.accumulate ? f[o] + fo : fo;
            t2 = fmaf(xf[c], xf[c], t2);
            vir = fmaf(xf[c], grad, vir);
        }
        // the k == i term contributed exp(0) = 1 and no force
        const float es = fp.A != 0.0 ? (esum.x - 1.0f) + esum.y : 0.f;
        v[0] = f2d_exact(fmaf(0.5f * om2, t2, 0.5f * (float)fp.A * es));
        v[1] = f2d_exact(vir);
    }
    block_reduce<2>(v, red);
    if (threadIdx.x == 0) {
        part[2 * (by * gx + bx) + 0] = v[0];
        part[2 * (by * gx + bx) + 1] = v[1];
    }
}

// Block-wide sums of NV double-float values per thread on the FP32 pipe (the
// FP64 pipe of this part is slow); the totals, as FP64, in `out` of thread 0.
// red: 2 * 32 * NV floats.
template <int NV>
__device__ __forceinline__ void block_reduce_df(df (&v)[NV], float* red, double (&out)[NV])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1)
            v[q] = df_add(v[q], df{__shfl_down_sync(0xffffffffu, v[q].h, o), __shfl_down_sync(0xffffffffu, v[q].l, o)});
    block_sync();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            red[2 * (w * NV + q)] = v[q].h;
            red[2 * (w * NV + q) + 1] = v[q].l;
        }
    block_sync();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            df t = lane < nw ? df{red[2 * (lane * NV + q)], red[2 * (lane * NV + q) + 1]} : df{0.f, 0.f};
            for (int o = 16; o > 0; o >>= 1)
                t = df_add(t, df{__shfl_down_sync(0xffffffffu, t.h, o), __shfl_down_sync(0xffffffffu, t.l, o)});
            if (lane == 0) out[q] = df2d(t);
        }
    }
    block_sync();
}

// (a1) + (a4) in mixed precision for one (slice j, particle block bx) unit,
// PT = blockDim.x particles: the springs and the trap + pair forces are summed
// in FP32 and stored once (overwriting F); the slice's spring energy (FP64
// differences, double-float squares and sums) and its trap + pair energy and
// virial (FP32 per particle, double-float sums) go to part_spr[j gx + bx] and
// part_pair[2 (j gx + bx)].  Same forces and energies as springs_unit followed
// by pair_unit_f32, with one FP32 rounding more on the force and no FP64
// arithmetic beyond one difference per coordinate.
template <int D, int PT>
__device__ __forceinline__ void force_unit_mixed(const BeadView& b, const ForceParams& fp, double* f, double* part_spr,
                                                 double* part_pair, int bx, int j, int gx, float2* sx, float* red)
{
    const int slot = j * gx + bx;
    if (bx * PT >= b.N) {  // a block past this replica's particles
        if (threadIdx.x == 0) {
            part_spr[slot] = 0.0;
            part_pair[2 * slot + 0] = 0.0;
            part_pair[2 * slot + 1] = 0.0;
        }
        return;
    }
    const int i = bx * PT + threadIdx.x;
    const size_t row = (size_t)D * b.ld;
    const double* rs = b.r + (size_t)j * row;
    const float sc = fp.sc32, ks = (float)fp.ks;
    float xf[D], fs[D];
    float2 xi[D], g[D];
    df es = df{0.f, 0.f};
#pragma unroll
    for (int c = 0; c < D; ++c) {
        xf[c] = 0.f;
        fs[c] = 0.f;
        if (i < b.N) {
            const double* p = rs + (size_t)c * b.ld + i;
            const double x = *p;
            const double xm = (j > 0) ? p[-(ptrdiff_t)row] : x;
            const double xp = (j < b.P - 1) ? p[row] : x;
            xf[c] = d2f_trunc(x);
            fs[c] = -ks * ((xf[c] - d2f_trunc(xm)) + (xf[c] - d2f_trunc(xp)));
            if (j < b.P - 1) {
                const df dd = d2df(xp - x);
                es = df_add(es, df_mul(dd, dd));
            }
        }
        const float xs = xf[c] * sc;
        xi[c] = make_float2(xs, xs);
        g[c] = make_float2(0.f, 0.f);
    }
    float2 esum = make_float2(0.f, 0.f);
    if (fp.A != 0.0) {
        for (int k0 = 0; k0 < b.N; k0 += PT) {
            const int k = k0 + threadIdx.x;
            float* sxf = reinterpret_cast<float*>(sx);
#pragma unroll
            for (int c = 0; c < D; ++c)
                sxf[c * PT + threadIdx.x] = (k < b.N) ? -d2f_trunc(rs[(size_t)c * b.ld + k]) * sc : -1.0e18f;
            __syncthreads();
            // partner pairs holding at least one particle (the padding past N
            // sits at -1e18 and adds exp2(-inf) = 0)
            const int nkk = (min(PT, b.N - k0) + 1) >> 1;
#pragma unroll 4
            for (int kk = 0; kk < nkk; ++kk) {
                float2 dx[D];
#pragma unroll
                for (int c = 0; c < D; ++c) dx[c] = __fadd2_rn(xi[c], sx[c * (PT / 2) + kk]);
                float2 q2 = __fmul2_rn(dx[0], dx[0]);
#pragma unroll
                for (int c = 1; c < D; ++c) q2 = __ffma2_rn(dx[c], dx[c], q2);
                const float2 ee = make_float2(ex2_approx(-q2.x), ex2_approx(-q2.y));
                esum = __fadd2_rn(esum, ee);
#pragma unroll
                for (int c = 0; c < D; ++c) g[c] = __ffma2_rn(ee, dx[c], g[c]);
            }
            __syncthreads();
        }
    }
    df v[3] = {es, df{0.f, 0.f}, df{0.f, 0.f}};
    if (i < b.N) {
        const float cpair = (float)fp.cpair32, om2 = (float)fp.omega2, mip = -(float)fp.inv_P;
        float t2 = 0.f, vir = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float grad = fmaf(om2, xf[c], cpair * (g[c].x + g[c].y));
            f[((size_t)j * D + c) * b.ld + i] = f2d_exact(fmaf(grad, mip, fs[c]));
            t2 = fmaf(xf[c], xf[c], t2);
            vir = fmaf(xf[c], grad, vir);
        }
        // the k == i term contributed exp(0) = 1 and no force
        const float es2 = fp.A != 0.0 ? (esum.x - 1.0f) + esum.y : 0.f;
        v[1] = df{fmaf(0.5f * om2, t2, 0.5f * (float)fp.A * es2), 0.f};
        v[2] = df{vir, 0.f};
    }
    double out[3];
    block_reduce_df<3>(v, red, out);
    if (threadIdx.x == 0) {
        part_spr[slot] = 0.5 * fp.ks * out[0];
        part_pair[2 * slot + 0] = out[1];
        part_pair[2 * slot + 1] = out[2];
    }
}

// ---------------------------------------------------------------------------
// Force work folded into the persistent exchange launch: the blocks after the
// chain and helper blocks take (slice, particle-block) units from a counter
// and compute the springs (overwriting F) and the trap + pairs (adding into
// F) of each unit.  They wait on nothing, so they only fill SMs the exchange
// recursion leaves idle.
struct ForceWork {
    BeadView b;
    ForceParams fp;      // accumulate is set per part
    double* part_spr;    // springs partials [gx * P]
    double* part_pair;   // pair partials [gx * P][2]
    int gx;              // particle blocks of blockDim.x per slice
    int* counter;        // next unit; zeroed before the launch
};

// Shared-memory bytes a force worker needs (blockDim.x = 256 particles).
constexpr int FW_SMEM = 16 + 96 * 8 + 3 * 256 * 8;

// `between` runs before each unit is claimed (every thread of the block; it
// may use the shared memory for other work and must leave it free).
template <int D, bool MIXED, class Between>
__device__ void force_worker_t(const ForceWork& w, unsigned char* smem, Between& between)
{
    constexpr int PT = 256;
    int* su = reinterpret_cast<int*>(smem);
    double* red = reinterpret_cast<double*>(smem + 16);  // [64] pairs, then [32] springs
    unsigned char* sx = smem + 16 + 96 * 8;
    const int nu = w.gx * w.b.P;
    ForceParams fs = w.fp, fq = w.fp;
    fs.accumulate = 0;
    fq.accumulate = 1;
    for (;;) {
        between();
        if (threadIdx.x == 0) *su = atomicAdd(w.counter, 1);
        block_sync();
        const int u = *su;
        block_sync();  // every thread has the unit before thread 0 takes the next
        if (u >= nu) break;
        const int j = u / w.gx, bx = u % w.gx;
        if (MIXED) {
            force_unit_mixed<D, PT>(w.b, w.fp, w.b.f, w.part_spr, w.part_pair, bx, j, w.gx, reinterpret_cast<float2*>(sx),
                                    reinterpret_cast<float*>(red));
        } else {
            springs_unit(w.b, fs, w.b.f, w.part_spr, bx, j, w.gx, red + 64);
            pair_unit_f64<D, PT>(w.b, fq, w.b.f, w.part_pair, bx, j, w.gx, reinterpret_cast<double*>(sx), red);
        }
        block_sync();  // the unit's shared memory is free for `between`
    }
}

template <class Between>
__device__ __forceinline__ void force_worker(const ForceWork& w, unsigned char* smem, Between& between)
{
    const bool mixed = w.fp.mixed != 0;
    if (w.b.d == 1) mixed ? force_worker_t<1, true>(w, smem, between) : force_worker_t<1, false>(w, smem, between);
    else if (w.b.d == 2) mixed ? force_worker_t<2, true>(w, smem, between) : force_worker_t<2, false>(w, smem, between);
    else mixed ? force_worker_t<3, true>(w, smem, between) : force_worker_t<3, false>(w, smem, between);
}
