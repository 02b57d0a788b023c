// Double-float exchange kernels (arXiv 2404.02628, Sec. III): prep, factor
// table, block operators, look-ahead recursion, band sums, endpoint forces.
// The equations are stated in pimd_xdf.cuh.
#include <math.h>
#include <stdio.h>

#include "pimd_xdf.cuh"

namespace {

// 32x32 dfw matrix.  Element (r, c) sits at RIDX(r, c): row r is rotated by
// r, so both row walks (lane = r) and column walks (lane = c) of a tile in
// shared memory hit 32 distinct banks, and a tile is one contiguous 4 KB run
// per component that cp.async copies verbatim.  Global tiles use the same order.
#define RIDX(r, c) (((r) << 5) + (((c) + (r)) & 31))
#define XDF_TILES 16  // tile slots per recursion block: 2 per helper warp, 2 x W for a chain block
struct DfwTile {
    float h[1024];
    float l[1024];
    int e[1024];
};

__device__ __forceinline__ void cp16(void* dst, const void* src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Asynchronous copy of a global tile into shared memory by `nthr` threads.
__device__ __forceinline__ void tile_copy(DfwTile* s, const float* h, const float* l, const int* e, int tid, int nthr)
{
    for (int q = tid; q < 256; q += nthr) {
        cp16(&s->h[4 * q], h + 4 * q);
        cp16(&s->l[4 * q], l + 4 * q);
        cp16(&s->e[4 * q], e + 4 * q);
    }
}

struct DVAcc {  // non-negative scalar s and signed vector v sharing exponent e
    df s;
    df v[3];
    int e;
};

__device__ __forceinline__ DVAcc dv_zero()
{
    DVAcc a;
    a.s = df{0.f, 0.f};
    a.v[0] = a.v[1] = a.v[2] = df{0.f, 0.f};
    a.e = WEF_ZERO_E;
    return a;
}

__device__ __forceinline__ void dv_renorm(DVAcc& a)
{
    if (!(a.s.h > 0.f)) return;
    const int ex = ((__float_as_int(a.s.h) >> 23) & 0xFF) - 127;
    if (ex == 0) return;
    const float f = pow2f(-ex);
    a.s = df_scale(a.s, f);
#pragma unroll
    for (int c = 0; c < 3; ++c) a.v[c] = df_scale(a.v[c], f);
    a.e += ex;
}

__device__ __forceinline__ void dv_add(DVAcc& A, const DVAcc& B)
{
    if (!(B.s.h > 0.f)) {
        if (B.s.h != 0.f) A.s = B.s;  // NaN propagates
        return;
    }
    if (!(A.s.h > 0.f)) {
        A = B;
        return;
    }
    const int E = max(A.e, B.e);
    const float fa = pow2f(A.e - E), fb = pow2f(B.e - E);
    A.s = df_add(df_scale(A.s, fa), df_scale(B.s, fb));
#pragma unroll
    for (int c = 0; c < 3; ++c) A.v[c] = df_add(df_scale(A.v[c], fa), df_scale(B.v[c], fb));
    A.e = E;
    dv_renorm(A);
}

// g(i,k) in double-float
__device__ __forceinline__ df xg(const XView& v, int i, int k)
{
    df s = df{0.f, 0.f};
    for (int c = 0; c < v.d; ++c) {
        const size_t oi = (size_t)c * v.npad + i, ok = (size_t)c * v.npad + k;
        const df x = df_sub(df{v.ah[oi], v.al[oi]}, df{v.bh[ok], v.bl[ok]});
        s = df_add(s, df_mul(x, x));
    }
    return df_mul(s, df{v.kap_h, v.kap_l});
}

// M[n][k] (zero outside 1 <= n <= N, k < n)
__device__ __forceinline__ dfw xM(const XView& v, int n, int k, const float2* tab)
{
    if (n < 1 || n > v.N || k >= n) return dfw_zero();
    const df x = df_sub(df{v.crh[n], v.crl[n]}, xg(v, n - 1, k));
    return dfw_exp(x, tab);
}

__device__ __forceinline__ dfw tile_get(const DfwTile* s, int r, int c)
{
    const int q = RIDX(r, c);
    return dfw{s->h[q], s->l[q], s->e[q]};
}
__device__ __forceinline__ void tile_put(DfwTile* s, int r, int c, dfw x)
{
    const int q = RIDX(r, c);
    s->h[q] = x.h;
    s->l[q] = x.l;
    s->e[q] = x.e;
}

// s += (a * f) * b for double-floats a, b and a power-of-two f: the product
// is split exactly (TwoProduct), the high parts summed with TwoSum, and all
// rounding errors collected in s.l (compensated dot product, Ogita-Rump-Oishi).
__device__ __forceinline__ void acc_term(df& s, float ah, float al, float bh, float bl, float f)
{
    ah = __fmul_rn(ah, f);
    al = __fmul_rn(al, f);
    const float p = __fmul_rn(ah, bh);
    const float pe = __fmaf_rn(ah, bh, -p);
    const float cross = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
    const df t = two_sum(s.h, p);
    s.h = t.h;
    s.l = __fadd_rn(s.l, __fadd_rn(t.l, __fadd_rn(pe, cross)));
}

// sum_{t in [t0,t1)} A[r][t] * x[t]  (x given as per-t dfw in shared arrays)
__device__ __forceinline__ dfw dot_row_vec(const DfwTile* A, int r, const float* xh, const float* xl, const int* xe,
                                           int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[RIDX(r, t)] + xe[t]);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int q = RIDX(r, t);
        acc_term(s, A->h[q], A->l[q], xh[t], xl[t], pow2f(A->e[q] + xe[t] - E));
    }
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// sum over t in [t0,t1) of A[r][t] * (x[t] + y[t])
__device__ __forceinline__ dfw dot_row_vec2(const DfwTile* A, int r, const float* xh, const float* xl, const int* xe,
                                            const float* yh, const float* yl, const int* ye, int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[RIDX(r, t)] + max(xe[t], ye[t]));
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int q = RIDX(r, t);
        acc_term(s, A->h[q], A->l[q], xh[t], xl[t], pow2f(A->e[q] + xe[t] - E));
        acc_term(s, A->h[q], A->l[q], yh[t], yl[t], pow2f(A->e[q] + ye[t] - E));
    }
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// sum over t in [t0,t1) of A[t][c] * (x[t] + y[t])
__device__ __forceinline__ dfw dot_col_vec2(const DfwTile* A, int c, const float* xh, const float* xl, const int* xe,
                                            const float* yh, const float* yl, const int* ye, int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[RIDX(t, c)] + max(xe[t], ye[t]));
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int q = RIDX(t, c);
        acc_term(s, A->h[q], A->l[q], xh[t], xl[t], pow2f(A->e[q] + xe[t] - E));
        acc_term(s, A->h[q], A->l[q], yh[t], yl[t], pow2f(A->e[q] + ye[t] - E));
    }
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// sum of n dfw values (max-exponent aligned compensated sum)
__device__ __forceinline__ dfw dfw_sum(const dfw* v, int n)
{
    int E = WEF_ZERO_E;
    for (int i = 0; i < n; ++i) E = max(E, v[i].e);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int i = 0; i < n; ++i) acc_term(s, v[i].h, v[i].l, 1.0f, 0.0f, pow2f(v[i].e - E));
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// sum_{t in [t0,t1)} A[t][c] * x[t]  (transposed)
__device__ __forceinline__ dfw dot_col_vec(const DfwTile* A, int c, const float* xh, const float* xl, const int* xe,
                                           int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[RIDX(t, c)] + xe[t]);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int q = RIDX(t, c);
        acc_term(s, A->h[q], A->l[q], xh[t], xl[t], pow2f(A->e[q] + xe[t] - E));
    }
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// (A B)[r][c] over t in [t0, t1)
__device__ __forceinline__ dfw dot_mat(const DfwTile* A, const DfwTile* B, int r, int c, int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[RIDX(r, t)] + B->e[RIDX(t, c)]);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int qa = RIDX(r, t), qb = RIDX(t, c);
        acc_term(s, A->h[qa], A->l[qa], B->h[qb], B->l[qb], pow2f(A->e[qa] + B->e[qb] - E));
    }
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// Weighted row sums of tile A for row r: s = sum_t A[r][t] w[t], v = sum_t A[r][t] w[t] u_c[t]
// where wu[c][t] = w[t].mant * u_c[t] (relative to w's exponent).
struct WeightSmem {
    float wh[32], wl[32];
    int we[32];
    float uh[3][32], ul[3][32];
};

__device__ __forceinline__ DVAcc weighted_rows(const DfwTile* A, const WeightSmem* w, int r, int d, int t0 = 0,
                                               int t1 = 32)
{
    DVAcc out = dv_zero();
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[RIDX(r, t)] + w->we[t]);
    if (E <= WEF_ZERO_E / 2) return out;
    for (int t = t0; t < t1; ++t) {
        const int q = RIDX(r, t);
        const float f = pow2f(A->e[q] + w->we[t] - E);
        const df a = df_scale(df{A->h[q], A->l[q]}, f);
        out.s = df_add(out.s, df_mul(a, df{w->wh[t], w->wl[t]}));
        for (int c = 0; c < d; ++c) out.v[c] = df_add(out.v[c], df_mul(a, df{w->uh[c][t], w->ul[c][t]}));
    }
    out.e = E;
    dv_renorm(out);
    return out;
}

__device__ __forceinline__ DVAcc weighted_cols(const DfwTile* A, const WeightSmem* w, int c0, int d, int t0 = 0,
                                               int t1 = 32)
{
    DVAcc out = dv_zero();
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[RIDX(t, c0)] + w->we[t]);
    if (E <= WEF_ZERO_E / 2) return out;
    for (int t = t0; t < t1; ++t) {
        const int q = RIDX(t, c0);
        const float f = pow2f(A->e[q] + w->we[t] - E);
        const df a = df_scale(df{A->h[q], A->l[q]}, f);
        out.s = df_add(out.s, df_mul(a, df{w->wh[t], w->wl[t]}));
        for (int c = 0; c < d; ++c) out.v[c] = df_add(out.v[c], df_mul(a, df{w->uh[c][t], w->ul[c][t]}));
    }
    out.e = E;
    dv_renorm(out);
    return out;
}

// Forward weights of column block I: y[k] and y[k] b_k (published by the chain).
__device__ __forceinline__ void load_wf(const XView& v, WeightSmem* w, int I, int lane)
{
    const int k = 32 * I + lane;
    w->wh[lane] = __ldcg(&v.yh[k]);
    w->wl[lane] = __ldcg(&v.yl[k]);
    w->we[lane] = __ldcg(&v.ye[k]);
    for (int c = 0; c < 3; ++c) {
        const bool on = c < v.d;
        w->uh[c][lane] = on ? __ldcg(&v.uh[(size_t)c * v.npad + k]) : 0.f;
        w->ul[c][lane] = on ? __ldcg(&v.ul[(size_t)c * v.npad + k]) : 0.f;
    }
}

// Backward weights of row block J: c[n] and c[n] a_{n-1} (published by the chain).
__device__ __forceinline__ void load_wb(const XView& v, WeightSmem* w, int J, int lane)
{
    const int n = 32 * J + lane;
    w->wh[lane] = __ldcg(&v.ch[n]);
    w->wl[lane] = __ldcg(&v.cl[n]);
    w->we[lane] = __ldcg(&v.ce[n]);
    for (int c = 0; c < 3; ++c) {
        const bool on = c < v.d;
        w->uh[c][lane] = on ? __ldcg(&v.wh[(size_t)c * v.npad + n]) : 0.f;
        w->ul[c][lane] = on ? __ldcg(&v.wl[(size_t)c * v.npad + n]) : 0.f;
    }
}

// Asynchronous copy of the published weights of block `blk` (forward: y and
// y b; backward: c and c a) into a weight slot, by one warp.
__device__ __forceinline__ void fetch_weights_warp(const XView& v, WeightSmem* w, int dir, int blk, int lane)
{
    const size_t o = (size_t)32 * blk;
    const float* h = dir == 0 ? v.yh : v.ch;
    const float* l = dir == 0 ? v.yl : v.cl;
    const int* e = dir == 0 ? v.ye : v.ce;
    const float* uh = dir == 0 ? v.uh : v.wh;
    const float* ul = dir == 0 ? v.ul : v.wl;
    const int nrows = 3 + 2 * v.d;  // 128-byte rows: wh, wl, we, then uh/ul per component
    for (int q = lane; q < nrows * 8; q += 32) {
        const int row = q >> 3, ch = (q & 7) * 4;
        const void* src;
        void* dst;
        if (row == 0) { src = h + o + ch; dst = w->wh + ch; }
        else if (row == 1) { src = l + o + ch; dst = w->wl + ch; }
        else if (row == 2) { src = e + o + ch; dst = w->we + ch; }
        else {
            const int c = (row - 3) >> 1;
            if (((row - 3) & 1) == 0) { src = uh + (size_t)c * v.npad + o + ch; dst = w->uh[c] + ch; }
            else { src = ul + (size_t)c * v.npad + o + ch; dst = w->ul[c] + ch; }
        }
        cp16(dst, src);
    }
}

// Columns [c0, c0+4) of tile (J,I) computed into shared memory (recompute mode).
__device__ __forceinline__ void compute_cols_warp(const XView& v, DfwTile* s, int J, int I, int c0, int lane,
                                                  const float2* tab)
{
    for (int c = c0; c < c0 + 4; ++c) tile_put(s, lane, c, xM(v, 32 * J + lane, 32 * I + c, tab));
}

// Rows [r0, r0+4) of tile (J,I) computed into shared memory (recompute mode).
__device__ __forceinline__ void compute_rows_warp(const XView& v, DfwTile* s, int J, int I, int r0, int lane,
                                                  const float2* tab)
{
    for (int r = r0; r < r0 + 4; ++r) tile_put(s, r, lane, xM(v, 32 * J + r, 32 * I + lane, tab));
}

__device__ __forceinline__ bool tile_stored(const XView& v, int J, int I) { return v.store || J - I < v.W; }

// Start the asynchronous copy of stored tile (J,I) by one warp (no-op for computed tiles).
__device__ __forceinline__ void fetch_tile_warp(const XView& v, DfwTile* s, int J, int I, int lane)
{
    if (!tile_stored(v, J, I)) return;
    const long long t = xdf_tile_index(v, J, I);
    tile_copy(s, v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024, lane, 32);
}

__device__ __forceinline__ size_t xpart_index(const XView& v, int dir, int blk, int s, int lane)
{
    return ((((size_t)dir * v.nb + blk) * v.S + s) << 5) + lane;
}
__device__ __forceinline__ size_t xband_index(const XView& v, int dir, int blk, int lane)
{
    return (((size_t)dir * v.nb + blk) << 5) + lane;
}

__device__ __forceinline__ void store_dv(float* h, float* l, int* e, size_t idx, const DVAcc& a)
{
    h[idx * 4] = a.s.h;
    l[idx * 4] = a.s.l;
    for (int c = 0; c < 3; ++c) {
        h[idx * 4 + 1 + c] = a.v[c].h;
        l[idx * 4 + 1 + c] = a.v[c].l;
    }
    e[idx] = a.e;
}

__device__ __forceinline__ DVAcc load_dv(const float* h, const float* l, const int* e, size_t idx)
{
    DVAcc a;
    a.s = df{__ldcg(&h[idx * 4]), __ldcg(&l[idx * 4])};
    for (int c = 0; c < 3; ++c) a.v[c] = df{__ldcg(&h[idx * 4 + 1 + c]), __ldcg(&l[idx * 4 + 1 + c])};
    a.e = __ldcg(&e[idx]);
    return a;
}

__device__ __forceinline__ void load_tab_smem(float2* tab_s, const float2* tab)
{
    for (int j = threadIdx.x; j < 256; j += blockDim.x) tab_s[j] = tab[j];
}

// ------------------------------------------------------------------------
// prep: double-float endpoints, row constants, link energy, flags

__global__ void __launch_bounds__(256) xdf_prep_kernel(XView v)
{
    __shared__ double red[64];
    double acc[2] = {0.0, 0.0};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < v.npad; q += gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            df a = df{0.f, 0.f}, b = df{0.f, 0.f};
            if (c < v.d && q < v.N) {
                a = df_from_double(v.a[(size_t)c * v.lda + q]);
                b = df_from_double(v.b[(size_t)c * v.ldb + q]);
            }
            v.ah[(size_t)c * v.npad + q] = a.h;
            v.al[(size_t)c * v.npad + q] = a.l;
            v.bh[(size_t)c * v.npad + q] = b.h;
            v.bl[(size_t)c * v.npad + q] = b.l;
        }
        // row constant of row n = q: c_n = g(n-1, n) - ln n - ln xi  (FP64, then split)
        df cr = df{0.f, 0.f};
        if (q >= 1 && q <= v.N) {
            double gl = 0.0;
            if (q < v.N)
                for (int c = 0; c < v.d; ++c) {
                    const double x = v.a[(size_t)c * v.lda + q - 1] - v.b[(size_t)c * v.ldb + q];
                    gl = fma(x, x, gl);
                }
            gl *= v.kappa;
            cr = df_from_double(gl - log((double)q) - v.log_xi);
        }
        v.crh[q] = cr.h;
        v.crl[q] = cr.l;
        if (q < v.N) {
            double gl = 0.0, gd = 0.0;
            for (int c = 0; c < v.d; ++c) {
                if (q < v.N - 1) {
                    const double x = v.a[(size_t)c * v.lda + q] - v.b[(size_t)c * v.ldb + q + 1];
                    gl = fma(x, x, gl);
                }
                const double y = v.a[(size_t)c * v.lda + q] - v.b[(size_t)c * v.ldb + q];
                gd = fma(y, y, gd);
            }
            gl *= v.kappa;
            gd *= v.kappa;
            acc[0] += gl;
            if (v.xi_zero) acc[1] += gl - log((double)(q + 1)) - gd;
        }
    }
    const int nflags = 2 * v.nb + 2 * v.nb * v.S;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nflags; j += gridDim.x * blockDim.x) v.flags[j] = 0;
    block_reduce<2>(acc, red);
    if (threadIdx.x == 0) {
        v.lsum[blockIdx.x * 2 + 0] = acc[0];
        v.lsum[blockIdx.x * 2 + 1] = acc[1];
    }
}

// ------------------------------------------------------------------------
// factor table: M tiles (all in store mode, band |J-I| < W otherwise)

__global__ void __launch_bounds__(256) xdf_table_kernel(XView v, long long ntiles)
{
    __shared__ float2 tab[256];
    load_tab_smem(tab, v.tab);
    block_sync();
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int J, I;
        if (v.store) {  // t = J(J+1)/2 + I; float estimate then integer correction
            J = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
            while ((long long)J * (J + 1) / 2 > t) --J;
            while ((long long)(J + 1) * (J + 2) / 2 <= t) ++J;
            I = (int)(t - (long long)J * (J + 1) / 2);
        } else {
            J = (int)(t / v.W);
            I = J - (int)(t % v.W);
        }
        float* Mh = v.Mh + t * 1024;
        float* Ml = v.Ml + t * 1024;
        int* Me = v.Me + t * 1024;
        for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
            const int r = q >> 5, c = q & 31;
            const dfw m = (I >= 0) ? xM(v, 32 * J + r, 32 * I + c, tab) : dfw_zero();
            const int o = RIDX(r, c);
            Mh[o] = m.h;
            Ml[o] = m.l;
            Me[o] = m.e;
        }
    }
}

// ------------------------------------------------------------------------
// block operators: G_J = (I - M_JJ)^{-1}, Q_J = G_J M_{J,J-1}, P_J = M_{J+1,J} G_J

__global__ void __launch_bounds__(256) xdf_blockops_kernel(XView v)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfwTile* L = reinterpret_cast<DfwTile*>(smem_raw);
    DfwTile* G = L + 1;
    DfwTile* Ms = L + 2;
    DfwTile* Mp = L + 3;
    const int J = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    {
        const long long t = xdf_tile_index(v, J, J);
        tile_copy(L, v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024, threadIdx.x, blockDim.x);
        if (J >= 1) {
            const long long ts = xdf_tile_index(v, J, J - 1);
            tile_copy(Ms, v.Mh + ts * 1024, v.Ml + ts * 1024, v.Me + ts * 1024, threadIdx.x, blockDim.x);
        }
        if (J + 1 < v.nb) {
            const long long tp = xdf_tile_index(v, J + 1, J);
            tile_copy(Mp, v.Mh + tp * 1024, v.Ml + tp * 1024, v.Me + tp * 1024, threadIdx.x, blockDim.x);
        }
        cp_commit();
        cp_wait<0>();
    }
    block_sync();
    // G = (I - L)^{-1} by forward substitution, one column per warp pass
    // (lane = row): after step t, lane t holds its final G[t][c], which is
    // broadcast and applied to the rows below.
    for (int c = w; c < 32; c += XDF_WARPS) {
        dfw acc = (lane == c) ? dfw{1.f, 0.f, 0} : dfw_zero();
        for (int t = c; t < 31; ++t) {
            dfw gt;
            gt.h = __shfl_sync(0xffffffffu, acc.h, t);
            gt.l = __shfl_sync(0xffffffffu, acc.l, t);
            gt.e = __shfl_sync(0xffffffffu, acc.e, t);
            if (lane > t) acc = dfw_add(acc, dfw_mul(tile_get(L, lane, t), gt));
        }
        tile_put(G, lane, c, (lane >= c) ? acc : dfw_zero());
    }
    block_sync();
    const size_t base = (size_t)J * 1024;
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
        const int r = q >> 5, c = q & 31, o = RIDX(r, c);
        v.Gh[base + o] = G->h[o];
        v.Gl[base + o] = G->l[o];
        v.Ge[base + o] = G->e[o];
        dfw Q = dfw_zero(), Pm = dfw_zero();
        if (J >= 1) Q = dot_mat(G, Ms, r, c, 0, r + 1);
        if (J + 1 < v.nb) Pm = dot_mat(Mp, G, r, c, c, 32);
        v.Qh[base + o] = Q.h;
        v.Ql[base + o] = Q.l;
        v.Qe[base + o] = Q.e;
        v.Ph[base + o] = Pm.h;
        v.Pl[base + o] = Pm.l;
        v.Pe[base + o] = Pm.e;
    }
}

// ------------------------------------------------------------------------
// recursion: chain blocks and helpers

struct ChainArrays {
    float xh[2][32], xl[2][32];   // solution blocks, x[J & 1] = block J (forward) / iteration parity (backward)
    int xe[2][32];
    float ghh[2][32], ghl[2][32]; // G h of the next block, double-buffered the same way
    int ghe[2][32];
    float hh[XDF_MAXW][32], hl[XDF_MAXW][32];  // band accumulators (ring, slot = block mod W)
    int he[XDF_MAXW][32];
    float ph[XDF_MAXW][32], pl[XDF_MAXW][32];  // helper partial sums (ring)
    int pe[XDF_MAXW][32];
    float rh[XDF_WARPS][32], rl[XDF_WARPS][32];  // per-warp partial results
    int re[XDF_WARPS][32];
};

struct ChainS {
    union {
        ChainArrays c;              // chain blocks
        DVAcc hm[XDF_WARPS][32];    // helper blocks: cross-warp merge
    } u;
    int abort;
    int ready;
    int y_ready, published, parts_ready, done;  // chain-block progress counters
    unsigned long long mb_all;                  // compute-warp barrier (6 arrivals)
    unsigned long long mb_pair[3];              // band warp-pair barriers (2 arrivals)
};

// Barrier for a subset of the warps of a block, on a shared-memory mbarrier:
// each warp reconverges, one lane arrives for it, and every lane waits for
// the phase to complete (bounded; a timeout records the error and raises the
// block's abort word).  `phase` is the warp's local count of completed uses.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* mb, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_sync(unsigned long long* mb, unsigned& phase, int lane, int limit, int* err,
                                          int* abort_word, int code)
{
    __syncwarp();
    if (lane == 0)
        asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_u32(mb)) : "memory");
    bool ok = false;
    for (int it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(smem_u32(mb)), "r"(phase & 1)
                     : "memory");
        if (done) {
            ok = true;
            break;
        }
    }
    phase += 1;
    if (!ok && lane == 0) {
        atomicCAS(err, 0, (PIMD_DEVERR_TIMEOUT << 24) | (code & 0xFFFFFF));
        *(volatile int*)abort_word = 1;
    }
    __syncwarp();
    return ok;
}

__device__ __forceinline__ dfw cget(const float (*h)[32], const float (*l)[32], const int (*e)[32], int i, int j)
{
    return dfw{h[i][j], l[i][j], e[i][j]};
}
__device__ __forceinline__ void cput(float (*h)[32], float (*l)[32], int (*e)[32], int i, int j, dfw x)
{
    h[i][j] = x.h;
    l[i][j] = x.l;
    e[i][j] = x.e;
}

// Tiles of iteration `it` by threads [0, nthr): forward T[0] = Q_J (G_0 first),
// T[1] = G_{J+1}, T[m] = M_{J+m,J}; backward T[0] = P_J (G_J first),
// T[1] = G_{J-1}, T[m] = M_{J,J-m}.
template <int DIR>
__device__ __forceinline__ void fetch_set_c(const XView& v, DfwTile* T, int it, int tid, int nthr)
{
    const int J = DIR == 0 ? it : v.nb - 1 - it;
    const size_t o = (size_t)J * 1024;
    if (it == 0) tile_copy(&T[0], v.Gh + o, v.Gl + o, v.Ge + o, tid, nthr);
    else if (DIR == 0) tile_copy(&T[0], v.Qh + o, v.Ql + o, v.Qe + o, tid, nthr);
    else tile_copy(&T[0], v.Ph + o, v.Pl + o, v.Pe + o, tid, nthr);
    const int Jn = DIR == 0 ? J + 1 : J - 1;
    if (Jn >= 0 && Jn < v.nb) {
        const size_t on = (size_t)Jn * 1024;
        tile_copy(&T[1], v.Gh + on, v.Gl + on, v.Ge + on, tid, nthr);
    }
    for (int m = 2; m < v.W; ++m) {
        const int Ja = DIR == 0 ? J + m : J, Ia = DIR == 0 ? J : J - m;
        if (DIR == 0 ? Ja < v.nb : Ia >= 0) {
            const long long t = xdf_tile_index(v, Ja, Ia);
            tile_copy(&T[m], v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024, tid, nthr);
        }
    }
    cp_commit();
}

// Shared-memory progress counters between the roles of a chain block.
__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ void vstore(int* p, int x) { *(volatile int*)p = x; }

// Bounded spin on a shared-memory counter; false if it gave up (recorded in
// the error word) or another role of the block has aborted.
__device__ __forceinline__ bool smem_wait_ge(const int* ctr, int want, ChainS* cs, int limit, int* err, int code)
{
    for (int it = 0; it < limit; ++it) {
        if (vload(ctr) >= want) {
            __threadfence_block();
            return true;
        }
        if (vload(&cs->abort)) return false;
        __nanosleep(32);
    }
    atomicCAS(err, 0, (PIMD_DEVERR_TIMEOUT << 24) | (code & 0xFFFFFF));
    vstore(&cs->abort, 1);
    return false;
}

template <int DIR>
__device__ __forceinline__ int chain_block(const XView& v, int it) { return DIR == 0 ? it : v.nb - 1 - it; }
template <int DIR>
__device__ __forceinline__ int chain_nparts(const XView& v, int B)
{
    return DIR == 0 ? min(v.S, B - v.W + 1) : min(v.S, v.nb - B - v.W);
}

// One chain block per direction.  Warps 0-5 compute; warp 6 fetches helper
// partials ahead of need; warp 7 publishes each solution block (values,
// weight products, release flag).  Compute iteration `it` (block J):
//   A: warps 0-3 critical partials of Q_J y_{J-1} (forward) / P_J^T c_{J+1}
//      (backward); warps 4-5 partials of G h (or G^T h) for the next block
//   B: warp 0 forms the block's solution; warp 4 forms the next G h;
//      warp 5 clears the consumed ring slots
//   C: warp pairs add the band tiles into the ring (W-2 tiles)
// The next iteration's tiles are copied during the current one.
template <int DIR>
__device__ void xchain(const XView& v, DfwTile* Tall, ChainS* cs)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int W = v.W, nb = v.nb;
    ChainArrays& C = cs->u.c;
    int* flag_chain = v.flags + DIR * nb;
    const int* flag_part = v.flags + 2 * nb + DIR * nb * v.S;
    const int lim = v.spin_limit;
    if (tid == 0) {
        cs->abort = 0;
        cs->y_ready = -1;
        cs->published = -1;
        cs->parts_ready = 0;
        cs->done = -1;
        mbar_init(&cs->mb_all, 6);
        for (int q = 0; q < 3; ++q) mbar_init(&cs->mb_pair[q], 2);
    }
    if (tid < 32) {
        for (int m = 0; m < W; ++m) {
            cput(C.hh, C.hl, C.he, m, tid, dfw_zero());
            cput(C.ph, C.pl, C.pe, m, tid, dfw_zero());
        }
        cput(C.ghh, C.ghl, C.ghe, 0, tid, dfw_zero());
        cput(C.ghh, C.ghl, C.ghe, 1, tid, dfw_zero());
    }
    block_sync();

    if (w == XDF_WARPS - 1) {
        // ---- publisher
        for (int it = 0; it < nb; ++it) {
            if (!smem_wait_ge(&cs->y_ready, it, cs, lim, v.err, 0x560000 + it)) break;
            const int J = chain_block<DIR>(v, it), xb = it & 1, n = 32 * J + lane;
            const df xm = df{C.xh[xb][lane], C.xl[xb][lane]};
            (DIR == 0 ? v.yh : v.ch)[n] = xm.h;
            (DIR == 0 ? v.yl : v.cl)[n] = xm.l;
            (DIR == 0 ? v.ye : v.ce)[n] = C.xe[xb][lane];
            for (int c = 0; c < v.d; ++c) {
                df u = df{0.f, 0.f};
                if (DIR == 0) u = df_mul(xm, df{v.bh[(size_t)c * v.npad + n], v.bl[(size_t)c * v.npad + n]});
                else if (n >= 1 && n <= v.N) u = df_mul(xm, df{v.ah[(size_t)c * v.npad + n - 1], v.al[(size_t)c * v.npad + n - 1]});
                (DIR == 0 ? v.uh : v.wh)[(size_t)c * v.npad + n] = u.h;
                (DIR == 0 ? v.ul : v.wl)[(size_t)c * v.npad + n] = u.l;
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                st_release(&flag_chain[J], 1);
                vstore(&cs->published, it);
            }
            __syncwarp();
        }
        return;
    }
    if (w == XDF_WARPS - 2) {
        // ---- helper-partial fetcher: the block of iteration it is needed for
        // the G h formed in iteration it-1; its ring slot is free once
        // iteration it-W-1 has finished.
        for (int it = 1; it < nb; ++it) {
            const int B = chain_block<DIR>(v, it), ns = chain_nparts<DIR>(v, B);
            if (ns > 0) {
                if (!smem_wait_ge(&cs->done, it - W - 1, cs, lim, v.err, 0x570000 + it)) break;
                int ok = 1;
                if (lane < ns) ok = wait_flag(&flag_part[B * v.S + lane], 1, v.err, lim, 0x510000 + (DIR << 16) + B);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) vstore(&cs->abort, 1);
                    __syncwarp();
                    break;
                }
                dfw t[8];
                for (int s = 0; s < ns; ++s) {
                    const size_t idx = xpart_index(v, DIR, B, s, lane);
                    t[s] = dfw{__ldcg(&v.parth[idx * 4]), __ldcg(&v.partl[idx * 4]), __ldcg(&v.parte[idx])};
                }
                for (int s = 0; s < ns; ++s) t[s] = dfw_norm(df{t[s].h, t[s].l}, t[s].e);
                cput(C.ph, C.pl, C.pe, B % W, lane, dfw_sum(t, ns));
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) vstore(&cs->parts_ready, it);
            __syncwarp();
        }
        return;
    }
    // ---- compute warps 0-5 (192 threads, named barrier 1; pairs use 2-4).
    // They never leave the loop early: after a failed wait (error recorded,
    // abort raised) they run to the end without waiting, so every named
    // barrier is met by all six warps.
    const int NCT = 6 * 32;
    unsigned ph_all = 0, ph_pair = 0;
    auto sync_all = [&](int code) { mbar_sync(&cs->mb_all, ph_all, lane, lim, v.err, &cs->abort, code); };
    fetch_set_c<DIR>(v, Tall, 0, tid, NCT);
    cp_wait<0>();
    sync_all(0x5a0000);
    for (int it = 0; it < nb; ++it) {
        const int J = chain_block<DIR>(v, it);
        DfwTile* T = Tall + (it & 1) * W;
        const bool more = it + 1 < nb;
        const int Jn1 = more ? chain_block<DIR>(v, it + 1) : 0;
        if (more) fetch_set_c<DIR>(v, Tall + ((it + 1) & 1) * W, it + 1, tid, NCT);
        const int xb = it & 1, pb = xb ^ 1;
        bool ok = true;
        // phase A
        if (w < 4) {
            if (it >= 1) {
                const dfw p = DIR == 0 ? dot_row_vec(&T[0], lane, C.xh[pb], C.xl[pb], C.xe[pb], 8 * w, 8 * w + 8)
                                       : dot_col_vec(&T[0], lane, C.xh[pb], C.xl[pb], C.xe[pb], 8 * w, 8 * w + 8);
                cput(C.rh, C.rl, C.re, w, lane, p);
            }
        } else if (more) {
            ok = smem_wait_ge(&cs->parts_ready, it + 1, cs, lim, v.err, 0x580000 + it);
            const int k = w - 4, s1 = Jn1 % W;
            dfw p = dfw_zero();
            if (ok) {
                if (DIR == 0) {
                    const int t0 = 16 * k, t1 = min(16 * k + 16, lane + 1);
                    if (t0 < t1) p = dot_row_vec2(&T[1], lane, C.hh[s1], C.hl[s1], C.he[s1], C.ph[s1], C.pl[s1], C.pe[s1], t0, t1);
                } else {
                    const int t0 = max(16 * k, lane), t1 = 16 * k + 16;
                    if (t0 < t1) p = dot_col_vec2(&T[1], lane, C.hh[s1], C.hl[s1], C.he[s1], C.ph[s1], C.pl[s1], C.pe[s1], t0, t1);
                }
            }
            cput(C.rh, C.rl, C.re, w, lane, p);
        }
        (void)ok;
        sync_all(0x5b0000 + it);
        // phase B
        if (w == 0) {
            // the slot x[xb] was last published two iterations ago
            ok = smem_wait_ge(&cs->published, it - 2, cs, lim, v.err, 0x590000 + it);
            dfw x;
            if (it == 0) {
                x = DIR == 0 ? tile_get(&T[0], lane, 0) : tile_get(&T[0], v.N - 32 * J, lane);
            } else {
                dfw t[5] = {cget(C.ghh, C.ghl, C.ghe, xb, lane), cget(C.rh, C.rl, C.re, 0, lane), cget(C.rh, C.rl, C.re, 1, lane),
                            cget(C.rh, C.rl, C.re, 2, lane), cget(C.rh, C.rl, C.re, 3, lane)};
                x = dfw_sum(t, 5);
            }
            cput(C.xh, C.xl, C.xe, xb, lane, x);
            __threadfence_block();
            __syncwarp();
            if (lane == 0) vstore(&cs->y_ready, it);
            __syncwarp();
        } else if (w == 4 && more) {
            dfw t[2] = {cget(C.rh, C.rl, C.re, 4, lane), cget(C.rh, C.rl, C.re, 5, lane)};
            cput(C.ghh, C.ghl, C.ghe, pb, lane, dfw_sum(t, 2));
        } else if (w == 5 && more) {
            const int s1 = Jn1 % W;
            cput(C.hh, C.hl, C.he, s1, lane, dfw_zero());
            cput(C.ph, C.pl, C.pe, s1, lane, dfw_zero());
        }
        sync_all(0x5c0000 + it);
        // phase C: band tiles (pairs of warps, one half of the columns each)
        if (w < 2 * (W - 2)) {
            const int m = 2 + (w >> 1), half = w & 1;
            const int Jt = DIR == 0 ? J + m : J - m;
            const bool on = DIR == 0 ? Jt < nb : Jt >= 0;
            if (on) {
                const dfw p = DIR == 0 ? dot_row_vec(&T[m], lane, C.xh[xb], C.xl[xb], C.xe[xb], 16 * half, 16 * half + 16)
                                       : dot_col_vec(&T[m], lane, C.xh[xb], C.xl[xb], C.xe[xb], 16 * half, 16 * half + 16);
                cput(C.rh, C.rl, C.re, w, lane, p);
            }
            mbar_sync(&cs->mb_pair[w >> 1], ph_pair, lane, lim, v.err, &cs->abort, 0x5d0000 + it);
            if (on && half == 0) {
                const int sl = Jt % W;
                dfw t[3] = {cget(C.hh, C.hl, C.he, sl, lane), cget(C.rh, C.rl, C.re, w, lane), cget(C.rh, C.rl, C.re, w + 1, lane)};
                cput(C.hh, C.hl, C.he, sl, lane, dfw_sum(t, 3));
            }
        }
        if (more) cp_wait<0>();
        sync_all(0x5e0000 + it);
        if (tid == 0) {
            __threadfence_block();
            vstore(&cs->done, it);
        }
        __syncwarp();
    }
    cp_wait<0>();
}

// Helper loop shared by both directions.  dir 0: items (B, s) = row block B,
// column blocks I = s, s+S, ... <= B-W (row sums).  dir 1: items (B, s) =
// column block B, row blocks J = B+W+s, B+W+s+S, ... < nb (column sums).
// All 8 warps work on every tile of an item, warp w on its 4 columns
// (forward) or rows (backward); tiles are visited from the first published
// to the last, copied one ahead (cp.async), and when the newest tile's flag
// is already set (checked once per item) no other flag is polled and the
// published weights are prefetched with the tile.
template <int DIR>
__device__ void xhelper(const XView& v, DfwTile* T, WeightSmem* Ws, ChainS* cs, const float2* tab, int h)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int* flag_chain = v.flags + DIR * v.nb;
    int* flag_part = v.flags + 2 * v.nb + DIR * v.nb * v.S;
    const int nh = DIR == 0 ? v.n_help_f : v.n_help_b;
    if (tid == 0) cs->abort = 0;
    block_sync();
    long long q = 0;
    for (int it = 0; it < v.nb; ++it) {
        const int B = DIR == 0 ? v.W + it : v.nb - 1 - v.W - it;
        if (DIR == 0 ? (B >= v.nb) : (B < 0)) break;
        const int ns = DIR == 0 ? min(v.S, B - v.W + 1) : min(v.S, v.nb - B - v.W);
        for (int si = 0; si < ns; ++si, ++q) {
            if (q % nh != h) continue;
            const int count = DIR == 0 ? (B - v.W - si) / v.S + 1 : (v.nb - 1 - (B + v.W + si)) / v.S + 1;
            // k-th tile in publication order: its other block index
            auto other = [&](int k) {
                return DIR == 0 ? si + k * v.S : B + v.W + si + (count - 1 - k) * v.S;
            };
            auto tJ = [&](int o) { return DIR == 0 ? B : o; };
            auto tI = [&](int o) { return DIR == 0 ? o : B; };
            if (tid == 0) cs->ready = ld_acquire(&flag_chain[other(count - 1)]) >= 1;
            {
                const int o0 = other(0);
                if (tile_stored(v, tJ(o0), tI(o0))) {
                    const long long t = xdf_tile_index(v, tJ(o0), tI(o0));
                    tile_copy(&T[0], v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024, tid, XDF_THREADS);
                }
            }
            block_sync();
            const bool all_ready = cs->ready != 0;
            if (all_ready && w == 0) fetch_weights_warp(v, &Ws[0], DIR, other(0), lane);
            cp_commit();
            DVAcc acc = dv_zero();
            bool aborted = false;
            for (int k = 0; k < count; ++k) {
                const int cur = k & 1, o = other(k);
                const int J = tJ(o), I = tI(o);
                if (k + 1 < count) {
                    const int on = other(k + 1);
                    if (tile_stored(v, tJ(on), tI(on))) {
                        const long long t = xdf_tile_index(v, tJ(on), tI(on));
                        tile_copy(&T[cur ^ 1], v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024, tid, XDF_THREADS);
                    }
                    if (all_ready && w == 0) fetch_weights_warp(v, &Ws[cur ^ 1], DIR, on, lane);
                }
                cp_commit();
                if (!all_ready) {
                    if (tid == 0) cs->ready = wait_flag(&flag_chain[o], 1, v.err, v.spin_limit, (DIR == 0 ? 0x530000 : 0x540000) + o);
                    block_sync();
                    if (!cs->ready) {
                        aborted = true;
                        break;
                    }
                    if (w == 0) {
                        if (DIR == 0) load_wf(v, &Ws[cur], I, lane);
                        else load_wb(v, &Ws[cur], J, lane);
                    }
                }
                cp_wait<1>();
                if (!tile_stored(v, J, I)) {
                    if (DIR == 0) compute_cols_warp(v, &T[cur], J, I, 4 * w, lane, tab);
                    else compute_rows_warp(v, &T[cur], J, I, 4 * w, lane, tab);
                }
                block_sync();
                const DVAcc p = DIR == 0 ? weighted_rows(&T[cur], &Ws[cur], lane, v.d, 4 * w, 4 * w + 4)
                                         : weighted_cols(&T[cur], &Ws[cur], lane, v.d, 4 * w, 4 * w + 4);
                dv_add(acc, p);
                block_sync();
            }
            cp_wait<0>();
            if (aborted) {
                if (tid == 0) cs->abort = 1;
                return;
            }
            cs->u.hm[w][lane] = acc;
            block_sync();
            if (w == 0) {
                DVAcc t = dv_zero();
                for (int q2 = 0; q2 < XDF_WARPS; ++q2) dv_add(t, cs->u.hm[q2][lane]);
                store_dv(v.parth, v.partl, v.parte, xpart_index(v, DIR, B, si, lane), t);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&flag_part[B * v.S + si], 1);
            }
            block_sync();
        }
    }
}

__global__ void __launch_bounds__(XDF_THREADS, 1) xdf_recursion_kernel(XView v)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfwTile* T = reinterpret_cast<DfwTile*>(smem_raw);
    WeightSmem* Ws = reinterpret_cast<WeightSmem*>(smem_raw + XDF_TILES * sizeof(DfwTile));
    ChainS* cs = reinterpret_cast<ChainS*>(smem_raw + XDF_TILES * sizeof(DfwTile) + XDF_WARPS * sizeof(WeightSmem));
    // the float2 table needs 8-byte alignment: round its offset up to 16 bytes
    const size_t tab_off = (XDF_TILES * sizeof(DfwTile) + XDF_WARPS * sizeof(WeightSmem) + sizeof(ChainS) + 15) & ~(size_t)15;
    float2* tab = reinterpret_cast<float2*>(smem_raw + tab_off);
    load_tab_smem(tab, v.tab);
    block_sync();
    const int bid = blockIdx.x;
    if (bid == 0) xchain<0>(v, T, cs);
    else if (bid == 1) xchain<1>(v, T, cs);
    else if (bid - 2 < v.n_help_f) xhelper<0>(v, T, Ws, cs, tab, bid - 2);
    else xhelper<1>(v, T, Ws, cs, tab, bid - 2 - v.n_help_f);
}

// Band sums: forward row block J over tiles I in [J-W+1, J]; backward column
// block I over row blocks [I, I+W-1].  One warp per tile, merged in order.
__global__ void __launch_bounds__(XDF_MAXW * 32) xdf_band_kernel(XView v)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfwTile* T = reinterpret_cast<DfwTile*>(smem_raw);
    WeightSmem* Ws = reinterpret_cast<WeightSmem*>(smem_raw + v.W * sizeof(DfwTile));
    DVAcc* hm = reinterpret_cast<DVAcc*>(smem_raw + v.W * (sizeof(DfwTile) + sizeof(WeightSmem)));
    __shared__ float2 tab[256];
    load_tab_smem(tab, v.tab);
    block_sync();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int blk = blockIdx.x, dir = blockIdx.y;
    DVAcc a = dv_zero();
    const int J = dir == 0 ? blk : blk + w, I = dir == 0 ? blk - w : blk;
    if (I >= 0 && J < v.nb) {
        fetch_tile_warp(v, &T[w], J, I, lane);
        cp_commit();
        if (dir == 0) load_wf(v, &Ws[w], I, lane);
        else load_wb(v, &Ws[w], J, lane);
        cp_wait<0>();
        __syncwarp();
        a = dir == 0 ? weighted_rows(&T[w], &Ws[w], lane, v.d) : weighted_cols(&T[w], &Ws[w], lane, v.d);
    }
    hm[w * 32 + lane] = a;
    block_sync();
    if (w == 0) {
        DVAcc t = dv_zero();
        for (int q = 0; q < v.W; ++q) dv_add(t, hm[q * 32 + lane]);
        store_dv(v.bandh, v.bandl, v.bande, xband_index(v, dir, blk, lane), t);
    }
}

__device__ __forceinline__ dfw xget(const float* h, const float* l, const int* e, int i) { return dfw{h[i], l[i], e[i]}; }

__device__ __forceinline__ double dv_comp(const DVAcc& a, int c, dfw scale)
{
    // a.v[c] * 2^a.e * scale
    dfw s = scale;
    s.e += a.e;
    return df_to_double(a.v[c]) * dfw_to_double(s);
}

// Endpoint forces (Sec. III exterior-bead formulas, factorised form).
__global__ void __launch_bounds__(256) xdf_finalize_kernel(XView v, FinalizeOut o)
{
    __shared__ double red[32];
    double esum[1] = {0.0};
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0 && v.lam) {
        if (v.xi_zero) {
            v.lam[0] = v.lam[1] = 0.0;
        } else {
            v.lam[0] = v.N * v.log_xi + dfw_log(xget(v.yh, v.yl, v.ye, v.N));
            v.lam[1] = v.N * v.log_xi + dfw_log(xget(v.ch, v.cl, v.ce, 0));
        }
    }
    if (l < v.N) {
        double a[3] = {0.0, 0.0, 0.0}, b[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < v.d; ++c) {
            a[c] = v.a[(size_t)c * v.lda + l];
            b[c] = v.b[(size_t)c * v.ldb + l];
        }
        double rowtot, coltot, PB[3] = {0.0, 0.0, 0.0}, PA[3] = {0.0, 0.0, 0.0}, link, linkin;
        if (v.xi_zero) {
            rowtot = coltot = 1.0;
            for (int c = 0; c < 3; ++c) {
                PB[c] = b[c];
                PA[c] = a[c];
            }
            link = linkin = 0.0;
        } else {
            const int n = l + 1;  // row of bead P of particle l
            const int Jn = n >> 5, rn = n & 31;
            const int Jk = l >> 5, rk = l & 31;
            DVAcc R = dv_zero(), C = dv_zero();
            for (int s = 0; s < min(v.S, Jn - v.W + 1); ++s) dv_add(R, load_dv(v.parth, v.partl, v.parte, xpart_index(v, 0, Jn, s, rn)));
            dv_add(R, load_dv(v.bandh, v.bandl, v.bande, xband_index(v, 0, Jn, rn)));
            for (int s = 0; s < min(v.S, v.nb - Jk - v.W); ++s) dv_add(C, load_dv(v.parth, v.partl, v.parte, xpart_index(v, 1, Jk, s, rk)));
            dv_add(C, load_dv(v.bandh, v.bandl, v.bande, xband_index(v, 1, Jk, rk)));
            const dfw Z = xget(v.yh, v.yl, v.ye, v.N);
            const double zm = df_to_double(df{Z.h, Z.l});
            const dfw iZ = dfw_norm(df_from_double(1.0 / zm), -Z.e);
            const dfw yn = xget(v.yh, v.yl, v.ye, n), cn = xget(v.ch, v.cl, v.ce, n);
            const dfw yl = xget(v.yh, v.yl, v.ye, l), cl = xget(v.ch, v.cl, v.ce, l);
            rowtot = dfw_to_double(dfw_mul(dfw_mul(yn, cn), iZ));
            coltot = dfw_to_double(dfw_mul(dfw_mul(yl, cl), iZ));
            const dfw fr = dfw_mul(cn, iZ), fc = dfw_mul(yl, iZ);
            for (int c = 0; c < v.d; ++c) {
                PB[c] = dv_comp(R, c, fr);
                PA[c] = dv_comp(C, c, fc);
            }
            link = (l < v.N - 1) ? 1.0 - rowtot : 0.0;
            linkin = (l >= 1) ? 1.0 - coltot : 0.0;
        }
        double FP[3], F1[3], e = 0.0;
        for (int c = 0; c < v.d; ++c) {
            const double bn = (l < v.N - 1) ? v.b[(size_t)c * v.ldb + l + 1] : 0.0;
            const double ap = (l >= 1) ? v.a[(size_t)c * v.lda + l - 1] : 0.0;
            FP[c] = -v.ks * (rowtot * a[c] - PB[c] + link * (a[c] - bn));
            F1[c] = -v.ks * (coltot * b[c] - PA[c] + linkin * (b[c] - ap));
            e += rowtot * a[c] * a[c] - 2.0 * a[c] * PB[c] + coltot * b[c] * b[c] + link * (a[c] - bn) * (a[c] - bn);
        }
        esum[0] = 0.5 * v.ks * e;
        if (o.f) {
            for (int c = 0; c < v.d; ++c) {
                o.f[((size_t)(o.P - 1) * v.d + c) * o.ldf + l] += FP[c];
                o.f[((size_t)c) * o.ldf + l] += F1[c];
            }
        }
        if (o.g1) {
            const double gs = *o.gscale;
            for (int c = 0; c < v.d; ++c) {
                o.g1[(size_t)c * o.ldg + l] = -gs * F1[c];
                o.gP[(size_t)c * o.ldg + l] = -gs * FP[c];
            }
        }
    }
    block_reduce<1>(esum, red);
    if (threadIdx.x == 0 && o.part) o.part[blockIdx.x] = esum[0];
}

}  // namespace

int xdf_prep_blocks(int npad) { return min(152, (npad + 255) / 256); }
int xdf_finalize_blocks(int N) { return (N + 255) / 256; }

size_t xdf_recursion_smem(int W)
{
    (void)W;
    const size_t tab_off = (XDF_TILES * sizeof(DfwTile) + XDF_WARPS * sizeof(WeightSmem) + sizeof(ChainS) + 15) & ~(size_t)15;
    return tab_off + 256 * sizeof(float2);
}

static size_t band_smem(int W) { return W * (sizeof(DfwTile) + sizeof(WeightSmem)) + W * 32 * sizeof(DVAcc); }
static size_t blockops_smem() { return 4 * sizeof(DfwTile); }

cudaError_t xdf_launch_forward(const XView& v, cudaStream_t st, ProfMarks* pm)
{
    xdf_prep_kernel<<<xdf_prep_blocks(v.npad), 256, 0, st>>>(v);
    prof_mark(pm, "exch_prep", st);
    if (v.xi_zero) return cudaGetLastError();
    const long long nt = xdf_ntiles(v.nb, v.W, v.store);
    const int tgrid = (int)min(nt, (long long)152 * 16);
    xdf_table_kernel<<<tgrid, 256, 0, st>>>(v, nt);
    prof_mark(pm, "exch_table", st);
    cudaError_t e;
    static bool attrs = false;
    if (!attrs) {
        e = cudaFuncSetAttribute(xdf_blockops_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)blockops_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(xdf_recursion_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)xdf_recursion_smem(XDF_MAXW));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(xdf_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem(XDF_MAXW));
        if (e != cudaSuccess) return e;
        attrs = true;
    }
    xdf_blockops_kernel<<<v.nb, 256, blockops_smem(), st>>>(v);
    prof_mark(pm, "exch_blockops", st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 + v.n_help_f + v.n_help_b);
    cfg.blockDim = dim3(XDF_THREADS);
    cfg.dynamicSmemBytes = xdf_recursion_smem(v.W);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, xdf_recursion_kernel, v);
    prof_mark(pm, "exch_recursion", st);
    return e;
}

cudaError_t xdf_launch_adjoint(const XView& v, const FinalizeOut& o, cudaStream_t st, ProfMarks* pm)
{
    if (!v.xi_zero) {
        xdf_band_kernel<<<dim3(v.nb, 2), 32 * v.W, band_smem(v.W), st>>>(v);
        prof_mark(pm, "exch_band", st);
    }
    xdf_finalize_kernel<<<xdf_finalize_blocks(v.N), 256, 0, st>>>(v, o);
    prof_mark(pm, "exch_finalize", st);
    return cudaGetLastError();
}

// 2^(j/256) as double-floats, from the host's long-double exp2 (>= 64-bit
// mantissa), uploaded once per workspace.
cudaError_t xdf_upload_table(float2* dev_table, cudaStream_t st)
{
    static float2 host_tab[256];
    static bool ready = false;
    if (!ready) {
        for (int j = 0; j < 256; ++j) {
            const long double x = exp2l((long double)j / 256.0L);
            const float h = (float)x;
            const float l = (float)(x - (long double)h);
            host_tab[j] = make_float2(h, l);
        }
        ready = true;
    }
    return cudaMemcpyAsync(dev_table, host_tab, sizeof(host_tab), cudaMemcpyHostToDevice, st);
}
