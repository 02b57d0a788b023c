// Springs (a1), trap + pairs (a4), NHC velocity Verlet (a5) and scalar
// reductions for sm_103a.
#include <algorithm>
#include <math.h>

#include "pimd_batch.cuh"
#include "pimd_forcework.cuh"

namespace {

constexpr int SPR_T = 128;
constexpr int MD_T = 256;



// ---------------------------------------------------------------------------
// (a1) Internal ring-polymer springs (Sec. III interior-bead formula and the
// within-particle half of the exterior-bead formulas): F_l^j = -k (2 r^j -
// r^{j+1} - r^{j-1}), with the missing neighbour of beads 1 and P dropped.
// Also sum_l E_int^(l) (always FP64).
__device__ __forceinline__ void springs_body(const BeadView& b, const ForceParams& fp, double* f, double* part)
{
    __shared__ double red[32];
    springs_unit(b, fp, f, part, blockIdx.x, blockIdx.y, gridDim.x, red);
}

__global__ void __launch_bounds__(SPR_T) springs_kernel(BeadView b, ForceParams fp, double* f, double* part)
{
    springs_body(b, fp, f, part);
}

// ---------------------------------------------------------------------------
// (a4) Trap + Gaussian pairs in each bead slice (Sec. II U, Sec. IV B):
// V_slice = sum_l 1/2 omega^2 r_l^2 + 1/2 sum_{i!=k} A exp(-|r_i - r_k|^2/s^2),
// F += -grad(V_slice)/P.  One thread per particle, the partner slice staged in
// shared memory 128 particles at a time.  Writes per-block (energy, virial).

template <int D, int PT>
__device__ __forceinline__ void pair_body_f64(const BeadView& b, const ForceParams& fp, double* f, double* part)
{
    __shared__ double sx[D * PT];
    __shared__ double red[64];
    pair_unit_f64<D, PT>(b, fp, f, part, blockIdx.x, blockIdx.y, gridDim.x, sx, red);
}

// FP32 pair arithmetic with exp2 on the MUFU unit; coordinates pre-scaled by
// sqrt(log2(e))/s so that each pair costs one ex2 and no extra multiply.
// One thread per particle; partners are taken two at a time on the packed
// FP32x2 pipe, the partner tile sitting in shared memory as negated
// coordinate pairs {x_k, x_k+1} per component.
template <int D, int PT>
__device__ __forceinline__ void pair_body_f32(const BeadView& b, const ForceParams& fp, double* f, double* part)
{
    __shared__ float2 sx[D * PT / 2];
    __shared__ double red[64];
    pair_unit_f32<D, PT>(b, fp, f, part, blockIdx.x, blockIdx.y, gridDim.x, sx, red);
}

template <int D, int PT>
__global__ void __launch_bounds__(PT) pair_kernel_f64(BeadView b, ForceParams fp, double* f, double* part)
{
    pair_body_f64<D, PT>(b, fp, f, part);
}

template <int D, int PT>
__global__ void __launch_bounds__(PT) pair_kernel_f32(BeadView b, ForceParams fp, double* f, double* part)
{
    pair_body_f32<D, PT>(b, fp, f, part);
}

// ---------------------------------------------------------------------------
// (a5) Massive Nose-Hoover chains (one chain of M thermostats of mass Q per
// degree of freedom) with the reversible Trotter half step of length tau:
// last link, links M-1..1 with exp(-tau/4 p_{k+1}/Q) scalings, the particle
// momentum scaled by exp(-tau p_1/Q), positions eta += tau p_eta/Q, then the
// links again in the opposite order.

__device__ __forceinline__ df dfc(const float (&c)[2]) { return df{c[0], c[1]}; }

// e^x for a double-float x, |x| <= 1/32: the Taylor series to x^4 in
// double-float (Horner form), the rest, x^5/120 (1 + x/6 + x^2/42 + x^3/336),
// in FP32 from the high part -- it is below 2.5e-10, so its FP32 rounding
// stays under 1e-16 -- and the truncation after x^8 below (1/32)^9/9! < 1e-19.
// The thermostat's arguments are of order 1e-3; larger |x| go through the
// FP64 library exp.
__device__ __forceinline__ df df_exp_small(df x)
{
    if (!(fabsf(x.h) <= 0.03125f)) return d2df(exp(df2d(x)));
#define PIMD_DFC(v) df{(float)(v), (float)((v) - (double)(float)(v))}
    const float xh = x.h;
    float t = fmaf(xh, 1.0f / 336.0f, 1.0f / 42.0f);
    t = fmaf(xh, t, 1.0f / 6.0f);
    t = fmaf(xh, t, 1.0f);
    t = xh * t * (1.0f / 120.0f);
    df s = df_add(PIMD_DFC(1.0 / 24.0), df{t, 0.f});
    s = df_add(df_mul(s, x), PIMD_DFC(1.0 / 6.0));
    s = df_add(df_mul(s, x), df{0.5f, 0.f});
    s = df_add(df_mul(s, x), df{1.f, 0.f});
    return df_add(df_mul(s, x), df{1.f, 0.f});
#undef PIMD_DFC
}

// One Trotter half step of length tau = dt/2 for the massive chains of one
// degree of freedom (Sec. IV A; MTK order): last link, links M-1..1 scaled by
// exp(-tau p_{k+1}/(4Q)), the momentum scaled by exp(-tau p_1/Q), eta drift,
// then the links again in reverse order.  Arithmetic in double-float on the
// FP32 pipe (FP64-accurate to about 1e-14); state read and written in FP64.
template <int M>
__device__ __forceinline__ void nhc_half_step(double& p64, double (&eta64)[M], double (&pe64)[M], const NhcConst& c)
{
    const df inv_m = dfc(c.inv_m), inv_Q = dfc(c.inv_Q), kT = df_neg(dfc(c.kT));
    const df ca = dfc(c.ca), cg = dfc(c.cg), ce = dfc(c.ce), cp = dfc(c.cp);
    df p = d2df(p64), q[M], e[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        q[k] = d2df(pe64[k]);
        e[k] = d2df(eta64[k]);
    }
    auto force = [&](int k) {  // G_k: kinetic energy of the link below, times 2, minus kT
        return df_add(k == 0 ? df_mul(df_mul(p, p), inv_m) : df_mul(df_mul(q[k - 1], q[k - 1]), inv_Q), kT);
    };
    q[M - 1] = df_add(q[M - 1], df_mul(cg, force(M - 1)));
#pragma unroll
    for (int k = M - 2; k >= 0; --k) {
        const df a = df_exp_small(df_mul(ca, q[k + 1]));
        q[k] = df_add(df_mul(q[k], df_mul(a, a)), df_mul(df_mul(cg, force(k)), a));
    }
    p = df_mul(p, df_exp_small(df_mul(cp, q[0])));
#pragma unroll
    for (int k = 0; k < M; ++k) e[k] = df_add(e[k], df_mul(ce, q[k]));
#pragma unroll
    for (int k = 0; k <= M - 2; ++k) {
        const df a = df_exp_small(df_mul(ca, q[k + 1]));
        q[k] = df_add(df_mul(q[k], df_mul(a, a)), df_mul(df_mul(cg, force(k)), a));
    }
    q[M - 1] = df_add(q[M - 1], df_mul(cg, force(M - 1)));
    p64 = df2d(p);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        pe64[k] = df2d(q[k]);
        eta64[k] = df2d(e[k]);
    }
}

// The same half step with the chain arithmetic in FP32 (mixed precision): the
// chain state is read and written in FP64, the momentum is scaled in FP64 by
// the FP32 factor.  e^x by the MUFU exp2 with the argument scaled by log2(e).
template <int M>
__device__ __forceinline__ void nhc_half_step_f32(double& p, double (&eta)[M], double (&pe)[M], float inv_m,
                                                  float inv_Q, float kT, float tau)
{
    const float L2E = 1.4426950408889634f;
    const float ca = -0.25f * tau * inv_Q * L2E, cg = 0.5f * tau, ce = tau * inv_Q;
    float q[M], e[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        q[k] = d2f_trunc(pe[k]);
        e[k] = d2f_trunc(eta[k]);
    }
    float pf = d2f_trunc(p);
    float G = ((M >= 2) ? q[M - 2] * q[M - 2] * inv_Q : pf * pf * inv_m) - kT;
    q[M - 1] = fmaf(cg, G, q[M - 1]);
#pragma unroll
    for (int k = M - 2; k >= 0; --k) {
        const float a = ex2_approx(ca * q[k + 1]);
        G = ((k == 0) ? pf * pf * inv_m : q[k - 1] * q[k - 1] * inv_Q) - kT;
        q[k] = fmaf(q[k], a * a, cg * G * a);
    }
    const float sp = ex2_approx(-tau * inv_Q * L2E * q[0]);
    p *= f2d_exact(sp);
    pf = d2f_trunc(p);
#pragma unroll
    for (int k = 0; k < M; ++k) e[k] = fmaf(ce, q[k], e[k]);
#pragma unroll
    for (int k = 0; k <= M - 2; ++k) {
        const float a = ex2_approx(ca * q[k + 1]);
        G = ((k == 0) ? pf * pf * inv_m : q[k - 1] * q[k - 1] * inv_Q) - kT;
        q[k] = fmaf(q[k], a * a, cg * G * a);
    }
    G = ((M >= 2) ? q[M - 2] * q[M - 2] * inv_Q : pf * pf * inv_m) - kT;
    q[M - 1] = fmaf(cg, G, q[M - 1]);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        pe[k] = f2d_exact(q[k]);
        eta[k] = f2d_exact(e[k]);
    }
}

// One degree of freedom: row (slice j, component c) = blockIdx.y, particle
// l = blockIdx.x * MD_T + threadIdx.x (a 2-D grid, so no index division).
template <bool PRE, int M>
__device__ __forceinline__ void md_body(const BeadView& b, const MDParams& mp)
{
    const int l = blockIdx.x * MD_T + threadIdx.x;
    if (l >= b.N || (int)blockIdx.y >= b.P * b.d) return;
    const size_t stride = (size_t)b.P * b.d * b.ld;
    const size_t o = (size_t)blockIdx.y * b.ld + l;
    double p = b.p[o];
    double eta[M], pe[M];
    if (mp.thermostat) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
            eta[k] = b.eta[k * stride + o];
            pe[k] = b.peta[k * stride + o];
        }
    }
    if (PRE) {
        if (mp.thermostat) {
            if (mp.nhc_fp32)
                nhc_half_step_f32<M>(p, eta, pe, mp.f_inv_mass, mp.f_inv_Q, mp.f_kT, mp.f_half_dt);
            else
                nhc_half_step<M>(p, eta, pe, mp.nc);
        }
        p = fma(mp.half_dt, b.f[o], p);
        b.r[o] = fma(mp.dt_inv_mass, p, b.r[o]);
    } else {
        p = fma(mp.half_dt, b.f[o], p);
        if (mp.thermostat) {
            if (mp.nhc_fp32)
                nhc_half_step_f32<M>(p, eta, pe, mp.f_inv_mass, mp.f_inv_Q, mp.f_kT, mp.f_half_dt);
            else
                nhc_half_step<M>(p, eta, pe, mp.nc);
        }
    }
    b.p[o] = p;
    if (mp.thermostat) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
            b.eta[k * stride + o] = eta[k];
            b.peta[k * stride + o] = pe[k];
        }
    }
}

template <bool PRE, int M>
__global__ void __launch_bounds__(MD_T) md_kernel(BeadView b, MDParams mp)
{
    md_body<PRE, M>(b, mp);
}

__device__ __forceinline__ void md_energy_body(const BeadView& b, const MDParams& mp, double* part)
{
    __shared__ double red[64];
    const size_t stride = (size_t)b.P * b.d * b.ld;
    double v[2] = {0.0, 0.0};
    for (size_t o = (size_t)blockIdx.x * MD_T + threadIdx.x; o < stride; o += (size_t)gridDim.x * MD_T) {
        const int l = (int)(o % b.ld);
        if (l >= b.N) continue;
        v[0] += 0.5 * b.p[o] * b.p[o] / mp.mass;
        if (mp.thermostat)
            for (int k = 0; k < b.M; ++k) {
                const double pe = b.peta[k * stride + o];
                v[1] += 0.5 * pe * pe / mp.Q + b.eta[k * stride + o] * mp.kT;
            }
    }
    block_reduce<2>(v, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = v[0];
        part[2 * blockIdx.x + 1] = v[1];
    }
}

__global__ void __launch_bounds__(MD_T) md_energy_kernel(BeadView b, MDParams mp, double* part)
{
    md_energy_body(b, mp, part);
}

// Fixed-order reduction of every per-block partial into the scalar slots.
__device__ __forceinline__ void scalars_body(const ScalarSources& s)
{
    double t[SC_COUNT];
    for (int q = 0; q < SC_COUNT; ++q) t[q] = 0.0;
    for (int i = 0; i < s.n_springs; ++i) t[SC_EINT] += s.springs[i];
    for (int sp = 0; sp < s.nsp; ++sp)
        for (int i = 0; i < s.n_lsum[sp]; ++i) {
            t[SC_GLINK] += s.lsum[sp][2 * i];
            t[SC_L0] += s.lsum[sp][2 * i + 1];
        }
    for (int i = 0; i < s.n_pair; ++i) {
        t[SC_U] += s.pair[2 * i];
        t[SC_VIRIAL] += s.pair[2 * i + 1];
    }
    for (int i = 0; i < s.n_fin; ++i) t[SC_SPRING_X] += s.fin[i];
    for (int i = 0; i < s.n_md; ++i) {
        t[SC_KIN] += s.md[2 * i];
        t[SC_THERMO] += s.md[2 * i + 1];
    }
    if (s.xi_zero) {
        t[SC_LAMBDA] = t[SC_L0];
        t[SC_LAMBDA_B] = t[SC_L0];
    } else {
        // the species' recursions are independent: their ln W_N add
        for (int sp = 0; sp < s.nsp; ++sp) {
            if (s.lam[sp]) {
                t[SC_LAMBDA] += s.lam[sp][0];
                t[SC_LAMBDA_B] += s.lam[sp][1];
            } else {
                const int n = s.N[sp];
                t[SC_LAMBDA] += n * s.log_xi + wef_log(Wef{s.y_m[sp][n], s.y_e[sp][n]});
                t[SC_LAMBDA_B] += n * s.log_xi + wef_log(Wef{s.c_m[sp][0], s.c_e[sp][0]});
            }
        }
    }
    for (int q = 0; q < SC_COUNT; ++q) s.out[q] = t[q];
}

__global__ void scalars_kernel(ScalarSources s)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    scalars_body(s);
}

// ---------------------------------------------------------------------------
// Batched wrappers: replica blockIdx.z, arguments from its RepArgs.

__global__ void __launch_bounds__(SPR_T) springs_batch(const RepArgs* ra)
{
    const RepArgs& a = ra[blockIdx.z];
    ForceParams fp = a.fp;
    fp.accumulate = 0;
    springs_body(a.bv, fp, a.bv.f, a.part_spr);
}

template <int D, bool MIXED, int PT>
__global__ void __launch_bounds__(PT) pair_batch(const RepArgs* ra)
{
    const RepArgs& a = ra[blockIdx.z];
    ForceParams fp = a.fp;
    fp.accumulate = 1;
    if (MIXED) pair_body_f32<D, PT>(a.bv, fp, a.bv.f, a.part_pair);
    else pair_body_f64<D, PT>(a.bv, fp, a.bv.f, a.part_pair);
}

template <bool PRE, int M>
__global__ void __launch_bounds__(MD_T) md_batch(const RepArgs* ra)
{
    const RepArgs& a = ra[blockIdx.z];
    md_body<PRE, M>(a.bv, a.mp);
}

// Springs and trap + pairs of every replica from the flat unit list (see
// ForceUnits): unit u of replica r covers slice j = k / gx_r and particles
// [bx PT, bx PT + PT), k = u - prefix[r], bx = k mod gx_r, gx_r = ceil(N_r / PT);
// partial sums go to slot j * fu.gx + bx.  Grid-stride, so the launch can be
// sized to leave room on every SM for the concurrent exchange step.
template <int D, bool MIXED, int PT>
__global__ void __launch_bounds__(PT) force_units_batch(const RepArgs* ra, ForceUnits fu)
{
    __shared__ double red[96];
    __shared__ __align__(16) unsigned char sx[D * PT * sizeof(double)];
    const int total = fu.prefix[fu.R];
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
        int lo = 0, hi = fu.R - 1;  // last replica whose first unit is <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (fu.prefix[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const RepArgs& a = ra[lo];
        const int gxr = (a.bv.N + PT - 1) / PT, k = u - fu.prefix[lo], j = k / gxr, bx = k - j * gxr;
        if (MIXED) {
            force_unit_mixed<D, PT>(a.bv, a.fp, a.bv.f, a.part_spr, a.part_pair, bx, j, fu.gx,
                                    reinterpret_cast<float2*>(sx), reinterpret_cast<float*>(red));
        } else {
            ForceParams fs = a.fp, fq = a.fp;
            fs.accumulate = 0;
            fq.accumulate = 1;
            springs_unit(a.bv, fs, a.bv.f, a.part_spr, bx, j, fu.gx, red + 64);
            pair_unit_f64<D, PT>(a.bv, fq, a.bv.f, a.part_pair, bx, j, fu.gx, reinterpret_cast<double*>(sx), red);
        }
        __syncthreads();  // shared scratch is reused by the next unit
    }
}

__global__ void __launch_bounds__(MD_T) md_energy_batch(const RepArgs* ra)
{
    const RepArgs& a = ra[blockIdx.z];
    md_energy_body(a.bv, a.mp, a.part_md);
}

__global__ void scalars_batch(const RepArgs* ra)
{
    if (threadIdx.x != 0) return;
    scalars_body(ra[blockIdx.x].ss);
}

__global__ void zero_kernel(double* x, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = 0.0;
}

__global__ void nonfinite_kernel(const double* x, int N, int P, int d, int ld, int* flag)
{
    const size_t n = (size_t)P * d * ld;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        if ((int)(o % ld) < N && !isfinite(x[o])) atomicOr(flag, 1);
}

}  // namespace

int springs_grid_x(int N) { return (N + SPR_T - 1) / SPR_T; }
int pair_grid_x(int N, int pt) { return (N + pt - 1) / pt; }
bool pair_block_ok(int pt) { return pt == 64 || pt == 128 || pt == 256; }
int md_blocks(int N, int P, int d)
{
    long long n = (long long)N * P * d;
    long long b = (n + MD_T - 1) / MD_T;
    return (int)(b < 152 * 8 ? b : 152 * 8);
}
// grid of the per-degree-of-freedom kernels: particles in x, (slice, component) rows in y
static dim3 md_grid(int N, int P, int d) { return dim3((N + MD_T - 1) / MD_T, P * d); }

cudaError_t launch_springs(const BeadView& b, const ForceParams& fp, double* f_out, double* part, cudaStream_t st)
{
    springs_kernel<<<dim3(springs_grid_x(b.N), b.P), SPR_T, 0, st>>>(b, fp, f_out, part);
    return cudaGetLastError();
}

template <int PT>
static void launch_pair_pt(const BeadView& b, const ForceParams& fp, double* f_out, double* part, cudaStream_t st)
{
    dim3 grid(pair_grid_x(b.N, PT), b.P);
    if (fp.mixed) {
        if (b.d == 1) pair_kernel_f32<1, PT><<<grid, PT, 0, st>>>(b, fp, f_out, part);
        else if (b.d == 2) pair_kernel_f32<2, PT><<<grid, PT, 0, st>>>(b, fp, f_out, part);
        else pair_kernel_f32<3, PT><<<grid, PT, 0, st>>>(b, fp, f_out, part);
    } else {
        if (b.d == 1) pair_kernel_f64<1, PT><<<grid, PT, 0, st>>>(b, fp, f_out, part);
        else if (b.d == 2) pair_kernel_f64<2, PT><<<grid, PT, 0, st>>>(b, fp, f_out, part);
        else pair_kernel_f64<3, PT><<<grid, PT, 0, st>>>(b, fp, f_out, part);
    }
}

cudaError_t launch_pair(const BeadView& b, const ForceParams& fp, double* f_out, double* part, cudaStream_t st, int pt)
{
    if (pt == 64) launch_pair_pt<64>(b, fp, f_out, part, st);
    else if (pt == 256) launch_pair_pt<256>(b, fp, f_out, part, st);
    else launch_pair_pt<128>(b, fp, f_out, part, st);
    return cudaGetLastError();
}

template <bool PRE>
static cudaError_t launch_md(const BeadView& b, const MDParams& mp, cudaStream_t st)
{
    const dim3 g = md_grid(b.N, b.P, b.d);
    switch (b.M) {
    case 1: md_kernel<PRE, 1><<<g, MD_T, 0, st>>>(b, mp); break;
    case 2: md_kernel<PRE, 2><<<g, MD_T, 0, st>>>(b, mp); break;
    case 3: md_kernel<PRE, 3><<<g, MD_T, 0, st>>>(b, mp); break;
    case 4: md_kernel<PRE, 4><<<g, MD_T, 0, st>>>(b, mp); break;
    case 5: md_kernel<PRE, 5><<<g, MD_T, 0, st>>>(b, mp); break;
    case 6: md_kernel<PRE, 6><<<g, MD_T, 0, st>>>(b, mp); break;
    case 7: md_kernel<PRE, 7><<<g, MD_T, 0, st>>>(b, mp); break;
    case 8: md_kernel<PRE, 8><<<g, MD_T, 0, st>>>(b, mp); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_md_pre(const BeadView& b, const MDParams& mp, cudaStream_t st) { return launch_md<true>(b, mp, st); }

cudaError_t launch_md_post(const BeadView& b, const MDParams& mp, cudaStream_t st) { return launch_md<false>(b, mp, st); }

cudaError_t launch_md_energy(const BeadView& b, const MDParams& mp, double* part, cudaStream_t st)
{
    md_energy_kernel<<<md_blocks(b.N, b.P, b.d), MD_T, 0, st>>>(b, mp, part);
    return cudaGetLastError();
}

cudaError_t launch_scalars(const ScalarSources& s, cudaStream_t st)
{
    scalars_kernel<<<1, 32, 0, st>>>(s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Seeded initial state (Sec. IV: beads drawn from a standard normal per
// coordinate, momenta from the Maxwell-Boltzmann distribution at kT = 1/beta).
// splitmix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator:
// output i of stream s mixes s + (i + 1) * 0x9E3779B97F4A7C15.  Coordinate
// (q, j, c, l) of quantity q (0: beads, 1: momenta) has counter
// k = ((q P + j) d + c) N + l and takes uniforms 2k and 2k + 1 in (0, 1]
// (top 53 bits, plus one unit); z = sqrt(-2 ln u1) cos(2 pi u2).

__host__ __device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i)
{
    return sm64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
}

__device__ __forceinline__ double sm64_uniform(unsigned long long seed, unsigned long long i)
{
    const unsigned long long x = sm64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
    return (double)((x >> 11) + 1ull) * 0x1.0p-53;
}

__global__ void __launch_bounds__(256) init_state_kernel(BeadView b, double p_scale, unsigned long long seed)
{
    const size_t n = (size_t)b.P * b.d * b.ld;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < 2 * n; o += (size_t)gridDim.x * blockDim.x) {
        const int q = o >= n ? 1 : 0;
        const size_t oq = o - q * n;
        const size_t row = oq / b.ld;  // j d + c
        const int l = (int)(oq - row * b.ld);
        double z = 0.0;
        if (l < b.N) {
            const unsigned long long k = ((unsigned long long)q * b.P * b.d + row) * b.N + l;
            const double u1 = sm64_uniform(seed, 2 * k), u2 = sm64_uniform(seed, 2 * k + 1);
            z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
        }
        if (q == 0) b.r[oq] = z;
        else b.p[oq] = p_scale * z;
    }
}

cudaError_t launch_init_state(const BeadView& b, double p_scale, unsigned long long seed, cudaStream_t st)
{
    const size_t n = 2 * (size_t)b.P * b.d * b.ld;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
    init_state_kernel<<<grid, 256, 0, st>>>(b, p_scale, seed);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Radial density of all beads (Sec. IV B density profiles, per particle):
// rho_b = n_b / (N P V_b).  Counts per block in shared memory, then one
// weighted atomic add per occupied bin.

__device__ __forceinline__ double shell_volume(int d, double r1, double r2)
{
    const double PI = 3.141592653589793;
    if (d == 1) return 2.0 * (r2 - r1);
    if (d == 2) return PI * (r2 * r2 - r1 * r1);
    return 4.0 / 3.0 * PI * (r2 * r2 * r2 - r1 * r1 * r1);
}

__global__ void __launch_bounds__(256) density_kernel(BeadView b, int nbins, double dr, double* hist)
{
    extern __shared__ unsigned int cnt[];
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) cnt[k] = 0u;
    __syncthreads();
    const long long n = (long long)b.P * b.N;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / b.N), l = (int)(q - (long long)j * b.N);
        double r2 = 0.0;
        for (int c = 0; c < b.d; ++c) {
            const double x = b.r[((size_t)j * b.d + c) * b.ld + l];
            r2 = __dadd_rn(r2, __dmul_rn(x, x));
        }
        const double t = floor(__ddiv_rn(__dsqrt_rn(r2), dr));
        if (t < (double)nbins) atomicAdd(&cnt[(int)t], 1u);
    }
    __syncthreads();
    const double inv = 1.0 / ((double)b.N * b.P);
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
        if (cnt[k]) atomicAdd(&hist[k], (double)cnt[k] * inv / shell_volume(b.d, k * dr, (k + 1) * dr));
}

cudaError_t launch_density(const BeadView& b, int nbins, double dr, double* hist, cudaStream_t st)
{
    if (nbins < 1 || nbins > DENSITY_MAX_BINS || !(dr > 0.0)) return cudaErrorInvalidValue;
    const long long n = (long long)b.P * b.N;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 4);
    const size_t smem = (size_t)nbins * sizeof(unsigned int);
    static DeviceOnce attr_once;
    const cudaError_t e = device_once(attr_once, [] {
        return cudaFuncSetAttribute(density_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(DENSITY_MAX_BINS * sizeof(unsigned int)));
    });
    if (e != cudaSuccess) return e;
    density_kernel<<<grid, 256, smem, st>>>(b, nbins, dr, hist);
    return cudaGetLastError();
}

cudaError_t launch_zero(double* x, size_t n, cudaStream_t st)
{
    zero_kernel<<<152, 256, 0, st>>>(x, n);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite_scan(const double* x, int N, int P, int d, int ld, int* flag, cudaStream_t st)
{
    nonfinite_kernel<<<152, 256, 0, st>>>(x, N, P, d, ld, flag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batched launchers

int batch_md_blocks(int nmax, int P, int d) { return (int)(((long long)nmax * P * d + MD_T - 1) / MD_T); }

cudaError_t batch_launch_md(const RepArgs* ra, const BatchGrid& g, bool pre, cudaStream_t st)
{
    const int M = g.M;
    const dim3 grid((g.nb_max * 32 + MD_T - 1) / MD_T, g.P * g.d, g.R);  // covers the largest replica
#define PIMD_MDB(m)                                                         \
    case m:                                                                 \
        if (pre) md_batch<true, m><<<grid, MD_T, 0, st>>>(ra);              \
        else md_batch<false, m><<<grid, MD_T, 0, st>>>(ra);                 \
        break;
    switch (M) {
        PIMD_MDB(1) PIMD_MDB(2) PIMD_MDB(3) PIMD_MDB(4) PIMD_MDB(5) PIMD_MDB(6) PIMD_MDB(7) PIMD_MDB(8)
    default: return cudaErrorInvalidValue;
    }
#undef PIMD_MDB
    return cudaGetLastError();
}

cudaError_t batch_launch_forces(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm)
{
    const int P = g.P, d = g.d;
    const bool mixed = g.mixed != 0;
    springs_batch<<<dim3(g.gx_spr, P, g.R), SPR_T, 0, st>>>(ra);
    prof_mark(pm, "batch_springs", st);
    const dim3 grid(g.gx_pair, P, g.R);
#define PIMD_PB(PT)                                                                 \
    if (mixed) {                                                                    \
        if (d == 1) pair_batch<1, true, PT><<<grid, PT, 0, st>>>(ra);               \
        else if (d == 2) pair_batch<2, true, PT><<<grid, PT, 0, st>>>(ra);          \
        else pair_batch<3, true, PT><<<grid, PT, 0, st>>>(ra);                      \
    } else {                                                                        \
        if (d == 1) pair_batch<1, false, PT><<<grid, PT, 0, st>>>(ra);              \
        else if (d == 2) pair_batch<2, false, PT><<<grid, PT, 0, st>>>(ra);         \
        else pair_batch<3, false, PT><<<grid, PT, 0, st>>>(ra);                     \
    }
    if (g.pair_t == 64) {
        PIMD_PB(64)
    } else if (g.pair_t == 256) {
        PIMD_PB(256)
    } else {
        PIMD_PB(128)
    }
#undef PIMD_PB
    prof_mark(pm, "batch_pair", st);
    return cudaGetLastError();
}

cudaError_t batch_launch_force_units(const RepArgs* ra, const ForceUnits& fu, const BatchGrid& g, int blocks,
                                     cudaStream_t st)
{
    const int d = g.d;
    const bool mixed = g.mixed != 0;
#define PIMD_FU(PT)                                                                         \
    if (mixed) {                                                                            \
        if (d == 1) force_units_batch<1, true, PT><<<blocks, PT, 0, st>>>(ra, fu);          \
        else if (d == 2) force_units_batch<2, true, PT><<<blocks, PT, 0, st>>>(ra, fu);     \
        else force_units_batch<3, true, PT><<<blocks, PT, 0, st>>>(ra, fu);                 \
    } else {                                                                                \
        if (d == 1) force_units_batch<1, false, PT><<<blocks, PT, 0, st>>>(ra, fu);         \
        else if (d == 2) force_units_batch<2, false, PT><<<blocks, PT, 0, st>>>(ra, fu);    \
        else force_units_batch<3, false, PT><<<blocks, PT, 0, st>>>(ra, fu);                \
    }
    if (g.pair_t == 64) {
        PIMD_FU(64)
    } else if (g.pair_t == 256) {
        PIMD_FU(256)
    } else {
        PIMD_FU(128)
    }
#undef PIMD_FU
    return cudaGetLastError();
}

cudaError_t batch_launch_scalars(const RepArgs* ra, const BatchGrid& g, cudaStream_t st)
{
    md_energy_batch<<<dim3(g.gx_md, 1, g.R), MD_T, 0, st>>>(ra);
    scalars_batch<<<g.R, 32, 0, st>>>(ra);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

static void split_df(double x, float (&out)[2])
{
    out[0] = (float)x;
    out[1] = (float)(x - (double)out[0]);
}

void nhc_constants(MDParams& mp)
{
    mp.half_dt = 0.5 * mp.dt;
    mp.dt_inv_mass = mp.dt * mp.inv_mass;
    const double tau = 0.5 * mp.dt;
    split_df(mp.inv_mass, mp.nc.inv_m);
    split_df(mp.inv_Q, mp.nc.inv_Q);
    split_df(mp.kT, mp.nc.kT);
    split_df(-0.25 * tau * mp.inv_Q, mp.nc.ca);
    split_df(0.5 * tau, mp.nc.cg);
    split_df(tau * mp.inv_Q, mp.nc.ce);
    split_df(-tau * mp.inv_Q, mp.nc.cp);
    mp.f_inv_mass = (float)mp.inv_mass;
    mp.f_inv_Q = (float)mp.inv_Q;
    mp.f_kT = (float)mp.kT;
    mp.f_half_dt = (float)tau;
}

void force_constants(ForceParams& fp, int P)
{
    fp.inv_P = 1.0 / P;
    fp.sc32 = (float)sqrt(fp.inv_s2 * 1.4426950408889634);
    fp.cpair32 = -2.0 * fp.A * fp.inv_s2 / (double)fp.sc32;
}
