// Double-float exchange kernels (arXiv 2404.02628, Sec. III): prep, factor
// table, block operators, look-ahead recursion, band sums, endpoint forces.
// The equations are stated in pimd_xdf.cuh.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "pimd_batch.cuh"
#include "pimd_forcework.cuh"

namespace {

// Element (r, c) of an XTile (see pimd_xdf.cuh).
#define RIDX(r, c) (((r) << 5) + (((c) + (r)) & 31))
#define XDF_TILES 16  // tile slots per recursion block: two per helper warp, a ring of 16 / W sets of W for a chain block
#define XDF_WSLOTS 16 // weight slots per recursion block: two per helper warp
typedef XTile DfwTile;

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
__device__ __forceinline__ void tile_copy(DfwTile* s, const XTile* g, int tid, int nthr)
{
    const float4* src = reinterpret_cast<const float4*>(g);
    float4* dst = reinterpret_cast<float4*>(s);
    for (int q = tid; q < (int)(sizeof(XTile) / 16); q += nthr) cp16(dst + q, src + q);
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

// Packed dfw for vectors in shared memory: {h, l, exponent bits, 0}, read
// by one 16-byte (broadcast) load.
__device__ __forceinline__ float4 dfw_pack(dfw x) { return make_float4(x.h, x.l, __int_as_float(x.e), 0.f); }
__device__ __forceinline__ dfw dfw_unpack(float4 x) { return dfw{x.x, x.y, __float_as_int(x.z)}; }

// sum over t in [c0, c1) of A[lane][t] x[t] (COL = false) or A[t][lane] x[t]
// (COL = true); c1 - c0 is a positive multiple of 8.  One pass: each 8-term
// chunk is loaded, its largest exponent taken, the running sum rescaled to
// the new largest exponent (a power of two: exact, or negligible when it
// underflows) and the chunk's terms added with the compensated acc_term.
template <bool COL>
__device__ __forceinline__ dfw dot_seg(const DfwTile* A, int lane, const float4* x, int c0, int c1)
{
    int E = WEF_ZERO_E;
    df s = df{0.f, 0.f};
    for (int t0 = c0; t0 < c1; t0 += 8) {
        float ah[8], al[8], xh[8], xl[8];
        int k[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = t0 + u, q = COL ? RIDX(t, lane) : RIDX(lane, t);
            const float4 xv = x[t];
            ah[u] = A->h[q];
            al[u] = A->l[q];
            xh[u] = xv.x;
            xl[u] = xv.y;
            k[u] = A->e[q] + __float_as_int(xv.z);
        }
        int Ec = k[0];
#pragma unroll
        for (int u = 1; u < 8; ++u) Ec = max(Ec, k[u]);
        const int En = max(E, Ec);
        const float g = pow2f(E - En);
        s.h = __fmul_rn(s.h, g);
        s.l = __fmul_rn(s.l, g);
        E = En;
#pragma unroll
        for (int u = 0; u < 8; ++u) acc_term(s, ah[u], al[u], xh[u], xl[u], pow2f(k[u] - E));
    }
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// sum of t[0..K) (max-exponent aligned compensated sum; zero entries add nothing)
template <int K>
__device__ __forceinline__ dfw dfw_sum_k(const dfw* t)
{
    int E = WEF_ZERO_E;
#pragma unroll
    for (int i = 0; i < K; ++i) E = max(E, t[i].e);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
#pragma unroll
    for (int i = 0; i < K; ++i) acc_term(s, t[i].h, t[i].l, 1.0f, 0.0f, pow2f(t[i].e - E));
    return dfw_norm(fast_two_sum(s.h, s.l), E);
}

// sum of t[0..n), n <= 8, with t[n..8) zero: the smallest fixed size that covers n
__device__ __forceinline__ dfw dfw_sum8(const dfw (&t)[8], int n)
{
    if (n <= 2) return dfw_sum_k<2>(t);
    if (n <= 4) return dfw_sum_k<4>(t);
    if (n <= 6) return dfw_sum_k<6>(t);
    return dfw_sum_k<8>(t);
}

// (A B)[r][c] over t in [t0, t1), both multiples of 8, in one pass: each
// 8-term chunk's largest exponent rescales the running sum as in dot_seg.
// Zero entries (exponent WEF_ZERO_E) add nothing, so the range may cover them.
__device__ __forceinline__ dfw dot_mat8(const DfwTile* A, const DfwTile* B, int r, int c, int t0, int t1)
{
    int E = WEF_ZERO_E;
    df s = df{0.f, 0.f};
    for (int tc = t0; tc < t1; tc += 8) {
        float ah[8], al[8], bh[8], bl[8];
        int k[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int qa = RIDX(r, tc + u), qb = RIDX(tc + u, c);
            ah[u] = A->h[qa];
            al[u] = A->l[qa];
            bh[u] = B->h[qb];
            bl[u] = B->l[qb];
            k[u] = A->e[qa] + B->e[qb];
        }
        int Ec = k[0];
#pragma unroll
        for (int u = 1; u < 8; ++u) Ec = max(Ec, k[u]);
        const int En = max(E, Ec);
        const float g = pow2f(E - En);
        s.h = __fmul_rn(s.h, g);
        s.l = __fmul_rn(s.l, g);
        E = En;
#pragma unroll
        for (int u = 0; u < 8; ++u) acc_term(s, ah[u], al[u], bh[u], bl[u], pow2f(k[u] - E));
    }
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
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
    tile_copy(s, v.M + t, lane, 32);
}

__device__ __forceinline__ size_t xpart_index(const XView& v, int dir, int blk, int s, int lane)
{
    return ((((size_t)dir * v.nb + blk) * v.S + s) << 5) + lane;
}
__device__ __forceinline__ size_t xband_index(const XView& v, int dir, int blk, int lane)
{
    return (((size_t)dir * v.nb + blk) << 5) + lane;
}
// the diagonal tile's sums (with the helper partials) sit after the band sums
__device__ __forceinline__ size_t xdiag_index(const XView& v, int dir, int blk, int lane)
{
    return (((size_t)(2 + dir) * v.nb + blk) << 5) + lane;
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

// (bx, gx): this block's index and the number of blocks sharing the work.
// FP64 -> double-float splits run on the integer pipe (d2df) and ln n comes
// from the workspace table, so the FP64 pipe does only the squared
// distances and the sums.
__device__ __forceinline__ void prep_body(const XView& v, int bx, int gx)
{
    __shared__ double red[64];
    double acc[2] = {0.0, 0.0};
    for (int q = bx * blockDim.x + threadIdx.x; q < v.npad; q += gx * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            df a = df{0.f, 0.f}, b = df{0.f, 0.f};
            if (c < v.d && q < v.N) {
                a = d2df(v.a[(size_t)c * v.lda + q]);
                b = d2df(v.b[(size_t)c * v.ldb + q]);
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
            cr = d2df(fma(gl, v.kappa, -v.lnn[q]) - v.log_xi);
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
            acc[0] = fma(gl, v.kappa, acc[0]);
            if (v.xi_zero) acc[1] += v.kappa * (gl - gd) - v.lnn[q + 1];
        }
    }
    const int nflags = 2 * v.nb + 2 * v.nb * v.S + 1;  // chain, partial flags, band-item counter
    for (int j = bx * blockDim.x + threadIdx.x; j < nflags; j += gx * blockDim.x) v.flags[j] = 0;
    block_reduce<2>(acc, red);
    if (threadIdx.x == 0) {
        v.lsum[bx * 2 + 0] = acc[0];
        v.lsum[bx * 2 + 1] = acc[1];
    }
}

__global__ void __launch_bounds__(256) xdf_prep_kernel(XView v) { prep_body(v, blockIdx.x, gridDim.x); }

// ------------------------------------------------------------------------
// factor table: M tiles (all in store mode, band |J-I| < W otherwise)

// One tile's factors M[n][k] = exp(c_n - kappa |a_{n-1} - b_k|^2): the 32 row
// endpoints a_{n-1}, row constants c_n and 32 column endpoints b_k are staged
// in shared memory once per tile; each element then needs only double-float
// arithmetic (difference, TwoProduct square, sum, scale) and the exp.
struct TableStage {
    float sa[3][2][32], sb[3][2][32], scr[2][32];
};

template <int D>
__device__ __forceinline__ void table_tile_t(const XView& v, long long t, const float2* tab, TableStage& st)
{
    const df kap = df{v.kap_h, v.kap_l};
    {
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
        block_sync();  // the previous tile's staged values are no longer read
        if (threadIdx.x < 32) {
            const int r = threadIdx.x, n = 32 * J + r;
            const bool on = n >= 1 && n <= v.N;
            for (int c = 0; c < 3; ++c) {
                const bool cc = on && c < v.d;
                st.sa[c][0][r] = cc ? v.ah[(size_t)c * v.npad + n - 1] : 0.f;
                st.sa[c][1][r] = cc ? v.al[(size_t)c * v.npad + n - 1] : 0.f;
            }
            st.scr[0][r] = on ? v.crh[n] : 0.f;
            st.scr[1][r] = on ? v.crl[n] : 0.f;
        } else if (threadIdx.x < 64 && I >= 0) {
            const int cl = threadIdx.x - 32, k = 32 * I + cl;
            for (int c = 0; c < 3; ++c) {
                const bool cc = c < v.d;
                st.sb[c][0][cl] = cc ? v.bh[(size_t)c * v.npad + k] : 0.f;
                st.sb[c][1][cl] = cc ? v.bl[(size_t)c * v.npad + k] : 0.f;
            }
        }
        block_sync();
        XTile* Mt = v.M + t;
        for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
            const int r = q >> 5, c = q & 31, n = 32 * J + r, k = 32 * I + c;
            dfw m = dfw_zero();
            if (I >= 0 && n >= 1 && n <= v.N && k < n) {
                df g = df{0.f, 0.f};
#pragma unroll
                for (int cc = 0; cc < D; ++cc) {
                    const df x = df_sub(df{st.sa[cc][0][r], st.sa[cc][1][r]}, df{st.sb[cc][0][c], st.sb[cc][1][c]});
                    df sq = two_prod(x.h, x.h);
                    sq.l = __fmaf_rn(2.f * x.h, x.l, sq.l);
                    g = df_add(g, sq);
                }
                m = dfw_exp(df_sub(df{st.scr[0][r], st.scr[1][r]}, df_mul(g, kap)), tab);
            }
            const int o = RIDX(r, c);
            Mt->h[o] = m.h;
            Mt->l[o] = m.l;
            Mt->e[o] = m.e;
        }
    }
}

template <int D>
__device__ __forceinline__ void table_body_t(const XView& v, long long ntiles, int bx, int gx)
{
    __shared__ float2 tab[256];
    __shared__ TableStage st;
    load_tab_smem(tab, v.tab);
    for (long long t = bx; t < ntiles; t += gx) table_tile_t<D>(v, t, tab, st);
}

// the dimension as a template argument, so the per-element coordinate loop unrolls
__device__ __forceinline__ void table_body(const XView& v, long long ntiles, int bx, int gx)
{
    if (v.d == 1) table_body_t<1>(v, ntiles, bx, gx);
    else if (v.d == 2) table_body_t<2>(v, ntiles, bx, gx);
    else table_body_t<3>(v, ntiles, bx, gx);
}

__global__ void __launch_bounds__(256) xdf_table_kernel(XView v, long long ntiles)
{
    table_body(v, ntiles, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------------
// block operators: G_J = (I - M_JJ)^{-1}, Q_J = G_J M_{J,J-1}, P_J = M_{J+1,J} G_J

// Two launches of 256-thread blocks: the substitution for eight columns of
// G_J (one column per warp), then a row quarter of Q_J = G_J M_{J,J-1} or
// P_J = M_{J+1,J} G_J (one entry per thread).  Many small blocks keep the
// SMs busy where one 1024-thread block per operator set left a third of
// them idle.
//
// G = (I - L)^{-1} by forward substitution, lane = row: after step t, lane t
// holds its final G[t][c], which is broadcast and applied to the rows below.
// Every entry is non-negative, so each lane keeps a compensated sum s
// relative to a running exponent E (s >= 1 once non-zero, far from the FP32
// limits) and adds one term per step; the raw (s, E) of lane t is what is
// broadcast.
__device__ __forceinline__ void blockops_g_item(const XView& v, int J, int gq, unsigned char* smem)
{
    DfwTile* L = reinterpret_cast<DfwTile*>(smem);
    const int tid = threadIdx.x, lane = tid & 31, c = 8 * gq + (tid >> 5);
    tile_copy(L, v.M + xdf_tile_index(v, J, J), tid, blockDim.x);
    cp_commit();
    cp_wait<0>();
    block_sync();
    df s = (lane == c) ? df{1.f, 0.f} : df{0.f, 0.f};
    int E = (lane == c) ? 0 : WEF_ZERO_E;
    for (int t = c; t < 31; ++t) {
        const float gh = __shfl_sync(0xffffffffu, s.h, t);
        const float gl = __shfl_sync(0xffffffffu, s.l, t);
        const int ge = __shfl_sync(0xffffffffu, E, t);
        if (lane > t) {
            const int q = RIDX(lane, t);
            const int k = L->e[q] + ge;
            if (k > E) {
                const float f = pow2f(E - k);
                s.h = __fmul_rn(s.h, f);
                s.l = __fmul_rn(s.l, f);
                E = k;
            }
            acc_term(s, L->h[q], L->l[q], gh, gl, pow2f(k - E));
        }
    }
    const int q = RIDX(lane, c);
    const dfw g = (lane >= c && E > WEF_ZERO_E / 2) ? dfw_norm(fast_two_sum(s.h, s.l), E) : dfw_zero();
    v.G[J].h[q] = g.h;
    v.G[J].l[q] = g.l;
    v.G[J].e[q] = g.e;
}

// Row quarter `qr` (rows 8 qr .. 8 qr + 7) of Q_J (part 0) or P_J (part 1);
// G_J has been published.
__device__ __forceinline__ void blockops_prod_item(const XView& v, int J, int part, int qr, unsigned char* smem)
{
    DfwTile* G = reinterpret_cast<DfwTile*>(smem);
    DfwTile* Mt = G + 1;
    const int tid = threadIdx.x;
    const bool on = part == 0 ? J >= 1 : J + 1 < v.nb;
    if (on) {
        tile_copy(G, v.G + J, tid, blockDim.x);
        tile_copy(Mt, v.M + (part == 0 ? xdf_tile_index(v, J, J - 1) : xdf_tile_index(v, J + 1, J)), tid, blockDim.x);
        cp_commit();
        cp_wait<0>();
    }
    block_sync();
    const int r = 8 * qr + (tid >> 5), c = tid & 31, o = RIDX(r, c);
    dfw x = dfw_zero();
    if (on) x = part == 0 ? dot_mat8(G, Mt, r, c, 0, (r + 8) & ~7) : dot_mat8(Mt, G, r, c, 0, 32);
    XTile* dst = (part == 0 ? v.Q : v.P) + J;
    dst->h[o] = x.h;
    dst->l[o] = x.l;
    dst->e[o] = x.e;
}

// grid (4, nb): part blockIdx.x of G_J, J = blockIdx.y
__global__ void __launch_bounds__(256) xdf_gparts_kernel(XView v)
{
    __shared__ __align__(16) unsigned char sm[sizeof(DfwTile)];
    blockops_g_item(v, blockIdx.y, blockIdx.x, sm);
}

// grid (8, nb): Q_J quarters 0-3, then P_J quarters 0-3, J = blockIdx.y
__global__ void __launch_bounds__(256) xdf_prods_kernel(XView v)
{
    __shared__ __align__(16) unsigned char sm[2 * sizeof(DfwTile)];
    blockops_prod_item(v, blockIdx.y, blockIdx.x >> 2, blockIdx.x & 3, sm);
}


// ------------------------------------------------------------------------
// recursion: chain blocks and helpers

#define XDF_XR 4        // solution blocks kept in shared memory (ring, slot = iteration mod XDF_XR)
#define XDF_NSETS 8     // most tile sets in flight (XDF_TILES / W)
#define XDF_NSEG 12     // phase-1 segments: two per compute warp
#define XDF_MAXS 8      // most helper partial streams per block

struct ChainArrays {
    float4 xv[XDF_XR + 1][32];                   // solution blocks (ring); slot XDF_XR: s = h + p of
                                                 // the block, the vector G acts on
    float hh[XDF_MAXW][32], hl[XDF_MAXW][32];    // band accumulators (ring, slot = block mod W)
    int he[XDF_MAXW][32];
    float ph[XDF_MAXW][32], pl[XDF_MAXW][32];    // helper partial sums (ring)
    int pe[XDF_MAXW][32];
    float4 r[XDF_NSEG][32];                      // phase-1 partial products, slot 2 w + j
};

struct ChainS {
    union {
        ChainArrays c;              // chain blocks
        DVAcc hm[XDF_WARPS][32];    // helper blocks: cross-warp merge
    } u;
    int abort;
    int ready;
    int y_ready, published, parts_ready, done;  // chain-block progress counters
    int seg_m[XDF_NSEG], seg_c0[XDF_NSEG], seg_c1[XDF_NSEG];  // phase-1 segments (m < 0: none)
    int red_idx[4][6], red_n[4];                // phase-2 sums: partial slots of warps 0-3
    unsigned long long mb_set[XDF_NSETS];       // tile-set arrival (bulk copies)
};

// the recursion block's dynamic shared memory (tiles, weight slots, chain or
// helper state, exp table) plus its static variables fit the 227 KB opt-in
static_assert(XDF_TILES * sizeof(DfwTile) + XDF_WSLOTS * sizeof(WeightSmem) + sizeof(ChainS) + 16 +
                      256 * sizeof(float2) + 64 <=
                  232448,
              "recursion block shared memory");

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* mb, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* mb, unsigned parity)
{
    unsigned done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done)
                 : "r"(smem_u32(mb)), "r"(parity & 1)
                 : "memory");
    return done != 0;
}

// Bounded wait for the completion of phase `parity` of a transaction
// barrier; gives up early once the block has aborted (unless `drain`, used
// to let every bulk copy land before the block exits).
__device__ __forceinline__ bool mbar_wait(unsigned long long* mb, unsigned parity, int limit, int* err, int* abort_word,
                                          int code, bool drain)
{
    for (int it = 0; it < limit; ++it) {
        if (mbar_test(mb, parity)) return true;
        if (!drain && (it & 63) == 63 && *(volatile int*)abort_word) return false;
    }
    atomicCAS(err, 0, (PIMD_DEVERR_TIMEOUT << 24) | (code & 0xFFFFFF));
    *(volatile int*)abort_word = 1;
    return false;
}

// Bulk (TMA, non-tensor) copy global -> shared, completing on an mbarrier.
// Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* mb)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mb))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
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

// Shared-memory progress counters between the roles of a chain block.
__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ void vstore(int* p, int x) { *(volatile int*)p = x; }

// Bounded spin on a shared-memory counter; false if it gave up (recorded in
// the error word) or another role of the block has aborted.
__device__ __forceinline__ bool smem_wait_ge(const int* ctr, int want, int* abort_word, int limit, int* err, int code)
{
    for (int it = 0; it < limit; ++it) {
        if (vload(ctr) >= want) {
            __threadfence_block();
            return true;
        }
        if (vload(abort_word)) return false;
        __nanosleep(32);
    }
    atomicCAS(err, 0, (PIMD_DEVERR_TIMEOUT << 24) | (code & 0xFFFFFF));
    vstore(abort_word, 1);
    return false;
}
__device__ __forceinline__ bool smem_wait_ge(const int* ctr, int want, ChainS* cs, int limit, int* err, int code)
{
    return smem_wait_ge(ctr, want, &cs->abort, limit, err, code);
}

template <int DIR>
__device__ __forceinline__ int chain_block(const XView& v, int it) { return DIR == 0 ? it : v.nb - 1 - it; }
template <int DIR>
__device__ __forceinline__ int chain_nparts(const XView& v, int B)
{
    return DIR == 0 ? min(v.S, B - v.W + 1) : min(v.S, v.nb - B - v.W);
}

// Tile m of iteration it (block J):
//   m = 0  Q_J (forward) / P_J (backward), times the previous solution block;
//   m = 1  G_J, times s_J = h_J + p_J;
//   m >= 2 band tile M_{J-1+m, J-1} (forward) / M_{J+1, J+1-m} (backward), times
//          the previous solution block, added into h of block J-1+m / J+1-m.
template <int DIR>
__device__ __forceinline__ bool chain_tile_on(const XView& v, int it, int m)
{
    if (m == 1) return true;
    if (it == 0) return false;
    if (m == 0) return true;
    const int J = chain_block<DIR>(v, it);
    return DIR == 0 ? J - 1 + m < v.nb : J + 1 - m >= 0;
}

// Phase-1 work split: the W tiles of an iteration are cut into 4W units of 8
// columns (rows), dealt in tile order to compute warps 0,4,1,5,2,3 in shares
// W/2, W-W/2, W/2, W-W/2, W, W, so that each of the four SM sub-partitions
// (warps w and w+4 share sub-partition w mod 4; warps 6 and 7 mostly wait)
// issues W units.  A share of at most 5 units spans at most two tiles.
__device__ __forceinline__ void chain_segments(int W, int* seg_m, int* seg_c0, int* seg_c1)
{
    const int order[6] = {0, 4, 1, 5, 2, 3};
    int u0 = 0;
    for (int k = 0; k < XDF_NSEG; ++k) seg_m[k] = -1;
    for (int q = 0; q < 6; ++q) {
        const int w = order[q];
        const int cnt = (q < 4) ? ((q & 1) ? W - W / 2 : W / 2) : W;
        const int u1 = u0 + cnt;
        int j = 0;
        for (int m = u0 >> 2; 4 * m < u1 && j < 2; ++m) {
            const int a = max(u0, 4 * m), b = min(u1, 4 * m + 4);
            if (a < b) {
                seg_m[2 * w + j] = m;
                seg_c0[2 * w + j] = 8 * (a - 4 * m);
                seg_c1[2 * w + j] = 8 * (b - 4 * m);
                ++j;
            }
        }
        u0 = u1;
    }
}

// Global source of tile m of iteration it (null if the tile is absent).
template <int DIR>
__device__ __forceinline__ const XTile* chain_tile_src(const XView& v, int it, int m)
{
    if (!chain_tile_on<DIR>(v, it, m)) return nullptr;
    const int J = chain_block<DIR>(v, it);
    if (m == 0) return (DIR == 0 ? v.Q : v.P) + J;
    if (m == 1) return v.G + J;
    return v.M + (DIR == 0 ? xdf_tile_index(v, J - 1 + m, J - 1) : xdf_tile_index(v, J + 1, J + 1 - m));
}

// Bulk copy of tile m of the set of iteration `it` into its ring slot: the
// set's mbarrier expects one arrival per tile slot (W), each with the bytes
// of its copy (none for an absent tile), so the copies of a set can be
// issued by different threads in any order.
template <int DIR>
__device__ __forceinline__ void chain_issue_tile(const XView& v, DfwTile* Tall, ChainS* cs, int it, int NS, int m)
{
    const int slot = it % NS;
    const XTile* src = chain_tile_src<DIR>(v, it, m);
    if (src) {
        mbar_expect_tx(&cs->mb_set[slot], (unsigned)sizeof(XTile));
        bulk_g2s(&Tall[slot * v.W + m], src, (unsigned)sizeof(XTile), &cs->mb_set[slot]);
    } else {
        asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_u32(&cs->mb_set[slot]))
                     : "memory");
    }
}

// Barrier of the six compute warps of a chain block (named barrier 1).
// bar.sync is warp-aligned, so each warp reconverges first.
__device__ __forceinline__ void compute_sync()
{
    __syncwarp();
    asm volatile("bar.sync 1, 192;" ::: "memory");
}

// One chain block per direction.  Warps 0-5 compute in two phases per
// iteration `it` (block J), separated by a barrier on those six warps:
//   1: every tile of the iteration's set times its vector (the previous
//      solution block, or s_J = h_J + p_J for G_J, which the G segments form
//      on their own entries first: the helper partial p_J is needed only
//      here), split into segments (chain_segments);
//   2: warp 0 sums the partials of Q_J y_{J-1} (P_J^T c_{J+1}) and G_J s_J into
//      the solution block; warps 1-3 add the band partials into the band
//      accumulators h of later blocks; warp 4 clears block J's h and p slots.
// Only phase 2 of warp 0 and phase 1 of the Q (P) segments lie on the
// dependent chain; the G s and band products for later blocks ride along.
// Warp 6 fetches helper partials ahead of need; warp 7 publishes each
// solution block (values, weight products, release flag) and then issues the
// bulk copy of a later tile set into the slot the block's phase 1 consumed.
template <int DIR>
__device__ void xchain(const XView& v, DfwTile* Tall, ChainS* cs)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int W = v.W, nb = v.nb, NS = XDF_TILES / W;
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
        chain_segments(W, cs->seg_m, cs->seg_c0, cs->seg_c1);
        // warp 0 sums tiles 0-1 (its block), warp r = 1..3 tile r+1 (band)
        for (int r = 0; r < 4; ++r) {
            const int mlo = r == 0 ? 0 : r + 1, mhi = r + 1;
            int n = 0;
            for (int k = 0; k < XDF_NSEG; ++k)
                if (cs->seg_m[k] >= mlo && cs->seg_m[k] <= mhi && n < 6) cs->red_idx[r][n++] = k;
            cs->red_n[r] = n;
        }
        for (int q = 0; q < NS; ++q) mbar_init(&cs->mb_set[q], W);  // one arrival per tile slot
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid < 32) {
        for (int m = 0; m < W; ++m) {
            cput(C.hh, C.hl, C.he, m, tid, dfw_zero());
            cput(C.ph, C.pl, C.pe, m, tid, dfw_zero());
        }
        C.xv[XDF_XR][tid] = dfw_pack(dfw_zero());
    }
    block_sync();

    if (w == XDF_WARPS - 1) {
        // ---- publisher and tile-set refills.  The endpoint coordinates of the
        // next block are loaded while the current one is awaited.  Every set of
        // the run is issued, also after an abort, so that every phase of every
        // slot completes.
        if (lane < W)
            for (int i = 0; i < min(NS, nb); ++i) chain_issue_tile<DIR>(v, Tall, cs, i, NS, lane);
        df e[3];
        auto load_e = [&](int it) {
            const int n = 32 * chain_block<DIR>(v, it) + lane;
            for (int c = 0; c < 3; ++c) {
                e[c] = df{0.f, 0.f};
                if (c >= v.d) continue;
                if (DIR == 0) e[c] = df{v.bh[(size_t)c * v.npad + n], v.bl[(size_t)c * v.npad + n]};
                else if (n >= 1 && n <= v.N) e[c] = df{v.ah[(size_t)c * v.npad + n - 1], v.al[(size_t)c * v.npad + n - 1]};
            }
        };
        load_e(0);
        bool ok = true;
        for (int it = 0; it < nb; ++it) {
            if (ok) ok = smem_wait_ge(&cs->y_ready, it, cs, lim, v.err, 0x560000 + it);
            if (ok) {
                const int J = chain_block<DIR>(v, it), xs = it % XDF_XR, n = 32 * J + lane;
                const dfw xw = dfw_unpack(C.xv[xs][lane]);
                const df xm = df{xw.h, xw.l};
                (DIR == 0 ? v.yh : v.ch)[n] = xm.h;
                (DIR == 0 ? v.yl : v.cl)[n] = xm.l;
                (DIR == 0 ? v.ye : v.ce)[n] = xw.e;
                for (int c = 0; c < v.d; ++c) {
                    const df u = df_mul(xm, e[c]);
                    (DIR == 0 ? v.uh : v.wh)[(size_t)c * v.npad + n] = u.h;
                    (DIR == 0 ? v.ul : v.wl)[(size_t)c * v.npad + n] = u.l;
                }
                // the warp barrier orders every lane's stores before lane 0's
                // release (cumulative), so one release publishes the block
                __syncwarp();
                if (lane == 0) {
                    st_release(&flag_chain[J], 1);
                    vstore(&cs->published, it);
                }
                __syncwarp();
                if (it + 1 < nb) load_e(it + 1);
            }
            // y of iteration it is ready, so phase 1 of iteration it -- the
            // only reader of its tile set -- is over: the slot takes the set of
            // it + NS once its previous copies have landed
            if (it + NS < nb) {
                if (lane == 0)
                    mbar_wait(&cs->mb_set[it % NS], (unsigned)(it / NS), lim, v.err, &cs->abort, 0x5f4000 + it, true);
                __syncwarp();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (lane < W) chain_issue_tile<DIR>(v, Tall, cs, it + NS, NS, lane);
            }
        }
        // every issued bulk copy lands before the block's shared memory is released
        if (lane == 0)
            for (int q = 0; q < NS && q < nb; ++q) {
                const int last = q + ((nb - 1 - q) / NS) * NS;
                mbar_wait(&cs->mb_set[q], (unsigned)(last / NS), lim, v.err, &cs->abort, 0x5f8000 + q, true);
            }
        return;
    }
    if (w == XDF_WARPS - 2) {
        // ---- helper-partial fetcher: the partials of the block of iteration
        // it are consumed in phase 1 of iteration it; its ring slot is cleared
        // in phase 2 of iteration it-W.
        // One global round trip per block in steady state: the flags of the
        // next block are polled (once, acquire) while this block's partials
        // are in flight, so a set flag needs no second round trip.
        int seen = 0;  // this lane's stream flag of the current block already observed set
        for (int it = 1; it < nb; ++it) {
            const int B = chain_block<DIR>(v, it), ns = chain_nparts<DIR>(v, B);
            if (ns > 0) {
                int ok = 1;
                if (lane < ns && !seen) ok = wait_flag(&flag_part[B * v.S + lane], 1, v.err, lim, 0x510000 + (DIR << 16) + B);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) vstore(&cs->abort, 1);
                    __syncwarp();
                    break;
                }
                __syncwarp();
                float ph8[8], pl8[8];
                int pe8[8];
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    ph8[s] = pl8[s] = 0.f;
                    pe8[s] = 0;
                    if (s < ns) {
                        const size_t idx = xpart_index(v, DIR, B, s, lane);
                        ph8[s] = __ldcg(&v.parth[idx * 4]);
                        pl8[s] = __ldcg(&v.partl[idx * 4]);
                        pe8[s] = __ldcg(&v.parte[idx]);
                    }
                }
                seen = 0;
                if (it + 1 < nb) {
                    const int B2 = chain_block<DIR>(v, it + 1), ns2 = chain_nparts<DIR>(v, B2);
                    if (lane < ns2) seen = ld_acquire(&flag_part[B2 * v.S + lane]) >= 1;
                }
                // the ring slot of block B was last read W iterations ago
                if (!smem_wait_ge(&cs->done, it - W, cs, lim, v.err, 0x570000 + it)) break;
                dfw t[8];
#pragma unroll
                for (int s = 0; s < 8; ++s) t[s] = s < ns ? dfw_norm(df{ph8[s], pl8[s]}, pe8[s]) : dfw_zero();
                cput(C.ph, C.pl, C.pe, B % W, lane, dfw_sum8(t, ns));
            } else {
                seen = 0;
                if (it + 1 < nb) {
                    const int B2 = chain_block<DIR>(v, it + 1), ns2 = chain_nparts<DIR>(v, B2);
                    if (lane < ns2) seen = ld_acquire(&flag_part[B2 * v.S + lane]) >= 1;
                }
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) vstore(&cs->parts_ready, it);
            __syncwarp();
        }
        return;
    }
    // ---- compute warps 0-5.  They never leave the loop early: after a
    // failed wait (error recorded, abort raised) they run to the end with
    // every further wait cut short, so the block always finishes.
    int sm[2], sc0[2], sc1[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        sm[j] = cs->seg_m[2 * w + j];
        sc0[j] = cs->seg_c0[2 * w + j];
        sc1[j] = cs->seg_c1[2 * w + j];
    }
    // phase-2 sums: partial slots of this warp's tiles
    int ridx[6], rn = 0;
    if (w <= 3) {
#pragma unroll
        for (int i = 0; i < 6; ++i) ridx[i] = cs->red_idx[w][i];
        rn = cs->red_n[w];
    }
    for (int it = 0; it < nb; ++it) {
        const int J = chain_block<DIR>(v, it), slot = it % NS;
        DfwTile* T = Tall + slot * W;
        mbar_wait(&cs->mb_set[slot], (unsigned)(it / NS), lim, v.err, &cs->abort, 0x5f0000 + it, false);
        // phase 1 (at it = 0 only warp 0 reads its block from G, before the
        // publisher may refill the slot once this iteration's y is ready)
        dfw x0 = dfw_zero();
        if (it == 0 && w == 0) x0 = DIR == 0 ? tile_get(&T[1], lane, 0) : tile_get(&T[1], v.N - 32 * J, lane);
        if (it >= 1) {
            const int xp = (it - 1) % XDF_XR;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int m = sm[j];
                if (m < 0) continue;
                dfw p = dfw_zero();
                if (chain_tile_on<DIR>(v, it, m)) {
                    if (m == 1) {
                        // s_J = h_J + p_J on this segment's entries (the helper
                        // partial of block J is needed only now)
                        smem_wait_ge(&cs->parts_ready, it, cs, lim, v.err, 0x580000 + it);
                        if (lane >= sc0[j] && lane < sc1[j]) {
                            const int sl = J % W;
                            C.xv[XDF_XR][lane] =
                                dfw_pack(dfw_add(cget(C.hh, C.hl, C.he, sl, lane), cget(C.ph, C.pl, C.pe, sl, lane)));
                        }
                        __syncwarp();
                    }
                    const float4* xv = C.xv[m == 1 ? XDF_XR : xp];
                    p = DIR == 0 ? dot_seg<false>(&T[m], lane, xv, sc0[j], sc1[j])
                                 : dot_seg<true>(&T[m], lane, xv, sc0[j], sc1[j]);
                }
                C.r[2 * w + j][lane] = dfw_pack(p);
            }
        }
        compute_sync();
        // phase 2
        if (w == 0) {
            // ring slot it % XDF_XR was last published XDF_XR iterations ago
            smem_wait_ge(&cs->published, it - XDF_XR, cs, lim, v.err, 0x590000 + it);
            dfw x = x0;
            if (it >= 1) {
                dfw t[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) t[i] = i < rn ? dfw_unpack(C.r[ridx[i < 6 ? i : 0]][lane]) : dfw_zero();
                x = dfw_sum8(t, rn);
            }
            C.xv[it % XDF_XR][lane] = dfw_pack(x);
            __threadfence_block();
            __syncwarp();
            if (lane == 0) vstore(&cs->y_ready, it);
            __syncwarp();
        } else if (w == 4) {
            // h and p of this block were read in phase 1: clear the slot for block J + W
            const int sl = J % W;
            cput(C.hh, C.hl, C.he, sl, lane, dfw_zero());
            cput(C.ph, C.pl, C.pe, sl, lane, dfw_zero());
        } else if (w <= 3) {
            const int m = w + 1;
            if (m < W && it >= 1 && chain_tile_on<DIR>(v, it, m)) {
                const int sl = (DIR == 0 ? J - 1 + m : J + 1 - m) % W;
                dfw t[8];
                t[0] = cget(C.hh, C.hl, C.he, sl, lane);
#pragma unroll
                for (int i = 0; i < 7; ++i) t[1 + i] = i < rn ? dfw_unpack(C.r[ridx[i < 6 ? i : 0]][lane]) : dfw_zero();
                cput(C.hh, C.hl, C.he, sl, lane, dfw_sum8(t, 1 + rn));
            }
        }
        compute_sync();
        if (tid == 0) {
            __threadfence_block();
            vstore(&cs->done, it);
        }
        __syncwarp();
    }
}

// Running weighted sums of one lane over the tiles of a helper item:
// s = sum_t A_t w_t and v_c = sum_t A_t u_{c,t}, where w_t is a published
// solution entry and u_{c,t} its product with an endpoint coordinate (same
// exponent as w_t).  Terms are scaled to the running largest exponent E;
// each 4-term chunk rescales the sums when E grows (powers of two: exact, or
// negligible when they underflow) and adds its terms with TwoSum /
// TwoProduct compensation.
struct RunAcc {
    df s, v[3];
    int E;
};

__device__ __forceinline__ void acc_prod(df& s, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    const float pe = __fmaf_rn(ah, bh, -p);
    const float cross = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
    const df t = two_sum(s.h, p);
    s.h = t.h;
    s.l = __fadd_rn(s.l, __fadd_rn(t.l, __fadd_rn(pe, cross)));
}

// All 32 terms of one tile for lane `lane`: row walk (COL = false, lane = row)
// or column walk (COL = true, lane = column).
// Terms [ta, ta + 4 * n4) of one tile (n4 chunks of 4 terms).
template <bool COL>
__device__ __forceinline__ void run_tile(RunAcc& ra, const DfwTile* A, const WeightSmem* w, int lane, int d, int ta = 0,
                                         int n4 = 8)
{
#pragma unroll 1
    for (int t0 = ta; t0 < ta + 4 * n4; t0 += 4) {
        float ah[4], al[4];
        int k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u, q = COL ? RIDX(t, lane) : RIDX(lane, t);
            ah[u] = A->h[q];
            al[u] = A->l[q];
            k[u] = A->e[q] + w->we[t];
        }
        int Ec = k[0];
#pragma unroll
        for (int u = 1; u < 4; ++u) Ec = max(Ec, k[u]);
        const int En = max(ra.E, Ec);
        const float g = pow2f(ra.E - En);
        ra.s = df_scale(ra.s, g);
#pragma unroll
        for (int c = 0; c < 3; ++c) ra.v[c] = df_scale(ra.v[c], g);
        ra.E = En;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u;
            const float f = pow2f(k[u] - En);
            const float a_h = __fmul_rn(ah[u], f), a_l = __fmul_rn(al[u], f);
            acc_prod(ra.s, a_h, a_l, w->wh[t], w->wl[t]);
            for (int c = 0; c < d; ++c) acc_prod(ra.v[c], a_h, a_l, w->uh[c][t], w->ul[c][t]);
        }
    }
}

__device__ __forceinline__ DVAcc run_to_dv(const RunAcc& ra)
{
    if (!(ra.s.h > 0.f) || ra.E <= WEF_ZERO_E / 2) {
        DVAcc z = dv_zero();
        if (ra.s.h != ra.s.h) z.s = ra.s;  // NaN propagates
        return z;
    }
    DVAcc out;
    out.s = fast_two_sum(ra.s.h, ra.s.l);
#pragma unroll
    for (int c = 0; c < 3; ++c) out.v[c] = fast_two_sum(ra.v[c].h, ra.v[c].l);
    out.e = ra.E;
    dv_renorm(out);
    return out;
}

// Helper loop shared by both directions.  dir 0: items (B, s) = row block B,
// column blocks I = s, s+S, ... <= B-W (row sums).  dir 1: items (B, s) =
// column block B, row blocks J = B+W+s, B+W+s+S, ... < nb (column sums).
// Tiles already published when the item starts go warp-per-tile (warp w
// takes tiles w, w+8, ..., all 32 terms per lane, one tile copied ahead with
// its weights; warp-local waits); the tiles still to come go through the whole
// block one by one as their flags are set (warp w on 4 columns / rows), which
// keeps the latency from the last publication to the partial short.  Both
// parts add into each warp's running sums; the eight warps' sums are merged
// in warp order and published with one release.
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
            // tiles [0, kr) were published when the item starts: flags are set
            // in publication order, so the published tiles form a prefix,
            // found by bisection
            if (tid == 0) {
                int lo = 0, hi = count;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (ld_acquire(&flag_chain[other(mid - 1)]) >= 1) lo = mid;
                    else hi = mid - 1;
                }
                cs->ready = lo;
            }
            block_sync();
            const int kr = cs->ready;
            RunAcc ra;
            ra.s = ra.v[0] = ra.v[1] = ra.v[2] = df{0.f, 0.f};
            ra.E = WEF_ZERO_E;
            bool ok = true;
            // part 1, throughput: warp w takes published tiles w, w+8, ...,
            // all 32 terms per lane, copied one tile ahead into its two slots
            auto issue = [&](int j) {
                const int k = w + XDF_WARPS * j;
                if (k < kr) {
                    const int o = other(k), sl = 2 * w + (j & 1);
                    if (tile_stored(v, tJ(o), tI(o))) {
                        const long long t = xdf_tile_index(v, tJ(o), tI(o));
                        tile_copy(&T[sl], v.M + t, lane, 32);
                    }
                    fetch_weights_warp(v, &Ws[sl], DIR, o, lane);
                }
                cp_commit();
            };
            issue(0);
            for (int j = 0; w + XDF_WARPS * j < kr; ++j) {
                const int k = w + XDF_WARPS * j, sl = 2 * w + (j & 1), o = other(k);
                const int J = tJ(o), I = tI(o);
                issue(j + 1);
                cp_wait<1>();
                __syncwarp();
                if (!tile_stored(v, J, I)) {
                    for (int c0 = 0; c0 < 32; c0 += 4) {
                        if (DIR == 0) compute_cols_warp(v, &T[sl], J, I, c0, lane, tab);
                        else compute_rows_warp(v, &T[sl], J, I, c0, lane, tab);
                    }
                    __syncwarp();
                }
                run_tile<DIR == 1>(ra, &T[sl], &Ws[sl], lane, v.d);
                __syncwarp();  // the slot is refilled by issue(j + 2)
            }
            cp_wait<0>();
            block_sync();
            // part 2, latency: the tiles still to be published, each by the
            // whole block (warp w on 4 of its columns / rows) as soon as its
            // flag is set; all of them copied at once (at most 16 per round)
            for (int k0 = kr; k0 < count; k0 += XDF_TILES) {
                const int nk = min(XDF_TILES, count - k0);
                for (int i = 0; i < nk; ++i) {
                    const int o = other(k0 + i);
                    if (tile_stored(v, tJ(o), tI(o))) {
                        const long long t = xdf_tile_index(v, tJ(o), tI(o));
                        tile_copy(&T[i], v.M + t, tid, XDF_THREADS);
                    }
                }
                cp_commit();
                for (int i = 0; i < nk && ok; ++i) {
                    const int o = other(k0 + i), J = tJ(o), I = tI(o), sl = i % XDF_WSLOTS;
                    if (tid == 0) cs->ready = wait_flag(&flag_chain[o], 1, v.err, v.spin_limit, (DIR == 0 ? 0x530000 : 0x540000) + o);
                    block_sync();
                    if (!cs->ready) {
                        ok = false;
                        break;
                    }
                    if (w == 0) {
                        if (DIR == 0) load_wf(v, &Ws[sl], I, lane);
                        else load_wb(v, &Ws[sl], J, lane);
                    }
                    cp_wait<0>();
                    if (!tile_stored(v, J, I)) {
                        if (DIR == 0) compute_cols_warp(v, &T[i], J, I, 4 * w, lane, tab);
                        else compute_rows_warp(v, &T[i], J, I, 4 * w, lane, tab);
                    }
                    block_sync();
                    run_tile<DIR == 1>(ra, &T[i], &Ws[sl], lane, v.d, 4 * w, 1);
                }
                cp_wait<0>();
                block_sync();
            }
            if (!ok && tid == 0) cs->abort = 1;
            cs->u.hm[w][lane] = run_to_dv(ra);
            block_sync();
            if (cs->abort) return;  // every thread reads it after the barrier
            // tree over the warps' sums (three levels), then warp 0 publishes
            for (int hs = 1; hs < XDF_WARPS; hs <<= 1) {
                if ((w & (2 * hs - 1)) == 0) {
                    DVAcc t = cs->u.hm[w][lane];
                    dv_add(t, cs->u.hm[w + hs][lane]);
                    cs->u.hm[w][lane] = t;
                }
                block_sync();
            }
            if (w == 0) {
                store_dv(v.parth, v.partl, v.parte, xpart_index(v, DIR, B, si, lane), cs->u.hm[0][lane]);
                __syncwarp();
                if (lane == 0) st_release(&flag_part[B * v.S + si], 1);
            }
            block_sync();
        }
    }
}

__device__ void band_worker(const XView& v);
__device__ void band_try(const XView& v);

__global__ void __launch_bounds__(XDF_THREADS, 1) xdf_recursion_kernel(XView v, ForceWork fw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfwTile* T = reinterpret_cast<DfwTile*>(smem_raw);
    WeightSmem* Ws = reinterpret_cast<WeightSmem*>(smem_raw + XDF_TILES * sizeof(DfwTile));
    ChainS* cs = reinterpret_cast<ChainS*>(smem_raw + XDF_TILES * sizeof(DfwTile) + XDF_WSLOTS * sizeof(WeightSmem));
    // the float2 table needs 8-byte alignment: round its offset up to 16 bytes
    const size_t tab_off = (XDF_TILES * sizeof(DfwTile) + XDF_WSLOTS * sizeof(WeightSmem) + sizeof(ChainS) + 15) & ~(size_t)15;
    float2* tab = reinterpret_cast<float2*>(smem_raw + tab_off);
    load_tab_smem(tab, v.tab);
    block_sync();
    const int bid = blockIdx.x;
    if (bid == 0) xchain<0>(v, T, cs);
    else if (bid == 1) xchain<1>(v, T, cs);
    else {
        if (bid - 2 < v.n_help_f) xhelper<0>(v, T, Ws, cs, tab, bid - 2);
        else if (bid - 2 - v.n_help_f < v.n_help_b) xhelper<1>(v, T, Ws, cs, tab, bid - 2 - v.n_help_f);
        else {
            // between force units, a band item whose inputs are published
            auto ready_band = [&v]() { band_try(v); };
            force_worker(fw, smem_raw, ready_band);
        }
        block_sync();
        band_worker(v);
    }
}

// Band sums: forward row block J over tiles I in [J-W+1, J]; backward column
// block I over row blocks [I, I+W-1], in two parts:
//   kind 0  the off-diagonal tiles (forward I < J, backward J > I), into the
//           band sums;
//   kind 1  the diagonal tile and the block's helper partials, into the
//           diagonal sums (the endpoint forces add the two);
//   kind -1 all tiles and partials into the band sums, the diagonal sums zero.
// The part's nt tiles are cut into nt H ranges of 32/H columns (forward) or
// rows (backward), H the largest power of two with nt H <= nw (nw = warps of
// the block); warp w takes ranges w, w + nw, ... and warp w adds helper
// partials w, w + nw, ...; a tree over the warps merges their sums.  With
// `wait` set, the first tiles are copied before thread 0 waits (bounded) for
// that flag, and the weights are read after it; false if the wait gave up.
__device__ __forceinline__ bool band_body(const XView& v, int blk, int dir, int kind, const int* wait = nullptr,
                                          int code = 0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_ok;
    const int nw = blockDim.x >> 5;
    DfwTile* T = reinterpret_cast<DfwTile*>(smem_raw);
    WeightSmem* Ws = reinterpret_cast<WeightSmem*>(smem_raw + nw * sizeof(DfwTile));
    DVAcc* hm = reinterpret_cast<DVAcc*>(smem_raw + nw * (sizeof(DfwTile) + sizeof(WeightSmem)));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blk >= v.nb) return true;  // a block past this replica's blocks
    const int m0 = kind == 0 ? 1 : 0, nt = (kind == 1 ? 1 : v.W) - m0;
    int H = 1;
    while (H < 32 && nt * 2 * H <= nw) H *= 2;
    const int span = 32 / H, nu = nt * H;
    int J = 0, I = 0, t0 = 0;
    auto fetch = [&](int u) {
        const int m = m0 + u / H;
        t0 = (u % H) * span;
        J = dir == 0 ? blk : blk + m;
        I = dir == 0 ? blk - m : blk;
        if (I < 0 || J >= v.nb) return false;
        fetch_tile_warp(v, &T[w], J, I, lane);
        cp_commit();
        return true;
    };
    bool have = w < nu && fetch(w);
    if (wait) {
        if (threadIdx.x == 0) s_ok = wait_flag(wait, 1, v.err, v.spin_limit, code);
        block_sync();
        if (!s_ok) {
            cp_wait<0>();  // the copies land before the shared memory is reused
            return false;
        }
    }
    DVAcc a = dv_zero();
    for (int u = w; u < nu;) {
        if (have) {
            if (dir == 0) load_wf(v, &Ws[w], I, lane);
            else load_wb(v, &Ws[w], J, lane);
            cp_wait<0>();
            __syncwarp();
            dv_add(a, dir == 0 ? weighted_rows(&T[w], &Ws[w], lane, v.d, t0, t0 + span)
                               : weighted_cols(&T[w], &Ws[w], lane, v.d, t0, t0 + span));
            __syncwarp();
        }
        u += nw;
        have = u < nu && fetch(u);
    }
    // the helper partials of the block were all released before the chain
    // formed the block, whose flag the caller waited for
    if (kind != 0) {
        const int ns = dir == 0 ? min(v.S, blk - v.W + 1) : min(v.S, v.nb - blk - v.W);
        for (int k = w; k < ns; k += nw)
            dv_add(a, load_dv(v.parth, v.partl, v.parte, xpart_index(v, dir, blk, k, lane)));
    }
    hm[w * 32 + lane] = a;
    block_sync();
    for (int h = 1; h < nw; h <<= 1) {
        if ((w & (2 * h - 1)) == 0 && w + h < nw) {
            DVAcc t = hm[w * 32 + lane];
            dv_add(t, hm[(w + h) * 32 + lane]);
            hm[w * 32 + lane] = t;
        }
        block_sync();
    }
    if (w == 0) {
        const size_t bi = xband_index(v, dir, blk, lane), di = xdiag_index(v, dir, blk, lane);
        store_dv(v.bandh, v.bandl, v.bande, kind == 1 ? di : bi, hm[lane]);
        if (kind == -1) store_dv(v.bandh, v.bandl, v.bande, di, dv_zero());
    }
    return true;
}

// Band items of the recursion launch, four per chain step it: forward and
// backward off-diagonal parts of the step's blocks (ready once the chain has
// published the block before), then their diagonal parts (ready once the
// block itself is published).  Their readiness is non-decreasing in u.
struct BandItem {
    int blk, dir, kind;
    const int* flag;  // chain flag to wait for (null: none)
};
__device__ __forceinline__ BandItem band_item(const XView& v, int u)
{
    BandItem b;
    const int it = u >> 2;
    b.dir = u & 1;
    b.kind = (u >> 1) & 1;
    b.blk = b.dir == 0 ? it : v.nb - 1 - it;
    const int src = b.kind == 1 ? b.blk : (b.dir == 0 ? b.blk - 1 : b.blk + 1);
    b.flag = (src >= 0 && src < v.nb) ? v.flags + b.dir * v.nb + src : nullptr;
    return b;
}

// Band sums inside the recursion launch: a force-worker block runs a band
// item whose inputs are already published between two force units
// (band_try); once its own work is done, a helper or force-worker block takes
// band items from the same counter in order, copying the item's tiles before
// waiting for its chain flag.  A wait that gives up ends the loop; the error
// word already holds the reason.
__device__ void band_worker(const XView& v)
{
    __shared__ int s_item;
    int* ctr = v.flags + 2 * v.nb + 2 * v.nb * v.S;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1);
        block_sync();
        const int u = s_item;
        if (u >= 4 * v.nb) break;
        const BandItem b = band_item(v, u);
        const bool ok = band_body(v, b.blk, b.dir, b.kind, b.flag, 0x5b0000 + u);
        block_sync();  // shared memory and s_item are reused by the next item
        if (!ok) break;
    }
}

// The next band item if its inputs are already published (no wait): claimed
// only by moving the counter from that item, so an item is never skipped.
__device__ void band_try(const XView& v)
{
    __shared__ int s_item;
    int* ctr = v.flags + 2 * v.nb + 2 * v.nb * v.S;
    if (threadIdx.x == 0) {
        int got = -1;
        const int u = *(volatile int*)ctr;
        if (u < 4 * v.nb) {
            const BandItem b = band_item(v, u);
            if ((!b.flag || ld_acquire(b.flag) >= 1) && atomicCAS(ctr, u, u + 1) == u) got = u;
        }
        s_item = got;
    }
    block_sync();
    const int u = s_item;
    if (u < 0) return;
    const BandItem b = band_item(v, u);
    band_body(v, b.blk, b.dir, b.kind);
    block_sync();
}

__device__ __forceinline__ dfw xget(const float* h, const float* l, const int* e, int i) { return dfw{h[i], l[i], e[i]}; }

// ln of a positive dfw, m 2^e with m = h + l in [1, 2): x0 = ln h in FP32,
// then one step of Newton's iteration for e^x = m taken to second order,
// ln m = x0 + t - t^2/2 with t = m e^{-x0} - 1 (|t| < 2^-20, so the neglected
// t^3/3 is below 2^-60), e^{-x0} by dfw_exp_core; FP64 only for the final
// e ln 2 + ln m.  The FP64 library logarithm costs microseconds of the FP64
// pipe on this part.
__device__ __forceinline__ double dfw_log_df(dfw a, const float2* tab)
{
    if (!(a.h > 0.0f)) return a.h == 0.0f ? -INFINITY : dfw_to_double(a);
    const float x0 = logf(a.h);
    const dfw ex = dfw_exp_core(df{-x0, 0.0f}, tab);
    const df p = df_scale(df_mul(df{a.h, a.l}, df{ex.h, ex.l}), pow2f(ex.e));
    const df t = df_sub(p, df{1.0f, 0.0f});
    const df lm = df_add(df{x0, 0.0f}, df_add(t, df{-0.5f * t.h * t.h, 0.0f}));
    const double ln2 = 0.6931471805599453;
    return fma((double)a.e, ln2, df_to_double(lm));
}


// x * 2^e as FP64 for a double-float x of any sign: the significand is built
// on the integer pipe (df2d) and e added into the exponent field while the
// result stays a normal double; zero, non-finite and out-of-range results
// take FP64 multiplications.
__device__ __forceinline__ double df_scaled_to_double(df x, int e)
{
    const double m = df2d(x);
    const long long bits = __double_as_longlong(m);
    const int E = (int)((bits >> 52) & 0x7FF);
    if (E > 0 && E < 0x7FF && E + e > 0 && E + e < 0x7FF) return __longlong_as_double(bits + ((long long)e << 52));
    if (m == 0.0 || E == 0x7FF) return m;
    if (e > 2000) return m * INFINITY;
    if (e < -2200) return m * 0.0;
    const int e1 = e / 2;
    return (m * pow2i(e1)) * pow2i(e - e1);
}

__device__ __forceinline__ double dfw_value(dfw a) { return df_scaled_to_double(df{a.h, a.l}, a.e); }

// a.v[c] * 2^a.e * scale, the product formed in double-float
__device__ __forceinline__ double dv_comp(const DVAcc& a, int c, dfw scale)
{
    return df_scaled_to_double(df_mul(a.v[c], df{scale.h, scale.l}), a.e + scale.e);
}

// 1 / Z for a non-zero dfw Z: the FP32 reciprocal of the high part refined by
// one Newton step in double-float (r + r (1 - z r)), about 2^-47 relative.
__device__ __forceinline__ dfw dfw_recip(dfw z)
{
    const float r0 = __frcp_rn(z.h);
    const df t = df_mul(df{z.h, z.l}, df{r0, 0.f});
    const df e1 = df_sub(df{1.f, 0.f}, t);
    const df r = df_add(df{r0, 0.f}, df_mul(df{r0, 0.f}, e1));
    return dfw_norm(r, -z.e);
}

// Endpoint forces (Sec. III exterior-bead formulas, factorised form).  D is
// the dimension (the coordinate loops unroll, nothing goes to local memory).
template <int D>
__device__ __forceinline__ void finalize_body(const XView& v, const FinalizeOut& o)
{
    __shared__ double red[32];
    double esum[1] = {0.0};
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    // ln Z of both directions, each on the first thread of its own block (the
    // FP64 logarithm is long on this part), the last block taking the second
    if (threadIdx.x == 0 && v.lam && (blockIdx.x == 0 || blockIdx.x == gridDim.x - 1)) {
        if (blockIdx.x == 0) v.lam[0] = v.xi_zero ? 0.0 : v.N * v.log_xi + dfw_log_df(xget(v.yh, v.yl, v.ye, v.N), v.tab);
        if (blockIdx.x == gridDim.x - 1)
            v.lam[1] = v.xi_zero ? 0.0 : v.N * v.log_xi + dfw_log_df(xget(v.ch, v.cl, v.ce, 0), v.tab);
    }
    if (l < v.N) {
        const int n = l + 1;  // row of bead P of particle l
        const int Jn = n >> 5, rn = n & 31;
        const int Jk = l >> 5, rk = l & 31;
        DVAcc R = dv_zero(), C = dv_zero();
        if (!v.xi_zero) {
            // band and diagonal sums (with the helper partials, band_body)
            R = load_dv(v.bandh, v.bandl, v.bande, xband_index(v, 0, Jn, rn));
            C = load_dv(v.bandh, v.bandl, v.bande, xband_index(v, 1, Jk, rk));
            dv_add(R, load_dv(v.bandh, v.bandl, v.bande, xdiag_index(v, 0, Jn, rn)));
            dv_add(C, load_dv(v.bandh, v.bandl, v.bande, xdiag_index(v, 1, Jk, rk)));
        }
        {
            double a[D], b[D];
            for (int c = 0; c < D; ++c) {
                a[c] = v.a[(size_t)c * v.lda + l];
                b[c] = v.b[(size_t)c * v.ldb + l];
            }
            double rowtot, coltot, PB[D], PA[D], link, linkin;
            if (v.xi_zero) {
                rowtot = coltot = 1.0;
                for (int c = 0; c < D; ++c) {
                    PB[c] = b[c];
                    PA[c] = a[c];
                }
                link = linkin = 0.0;
            } else {
                const dfw iZ = dfw_recip(xget(v.yh, v.yl, v.ye, v.N));
                const dfw yn = xget(v.yh, v.yl, v.ye, n), cn = xget(v.ch, v.cl, v.ce, n);
                const dfw yl = xget(v.yh, v.yl, v.ye, l), cl = xget(v.ch, v.cl, v.ce, l);
                rowtot = dfw_value(dfw_mul(dfw_mul(yn, cn), iZ));
                coltot = dfw_value(dfw_mul(dfw_mul(yl, cl), iZ));
                const dfw fr = dfw_mul(cn, iZ), fc = dfw_mul(yl, iZ);
                for (int c = 0; c < D; ++c) {
                    PB[c] = dv_comp(R, c, fr);
                    PA[c] = dv_comp(C, c, fc);
                }
                link = (l < v.N - 1) ? 1.0 - rowtot : 0.0;
                linkin = (l >= 1) ? 1.0 - coltot : 0.0;
            }
            double FP[D], F1[D], e = 0.0;
            for (int c = 0; c < D; ++c) {
                const double bn = (l < v.N - 1) ? v.b[(size_t)c * v.ldb + l + 1] : 0.0;
                const double ap = (l >= 1) ? v.a[(size_t)c * v.lda + l - 1] : 0.0;
                FP[c] = -v.ks * (rowtot * a[c] - PB[c] + link * (a[c] - bn));
                F1[c] = -v.ks * (coltot * b[c] - PA[c] + linkin * (b[c] - ap));
                e += rowtot * a[c] * a[c] - 2.0 * a[c] * PB[c] + coltot * b[c] * b[c] + link * (a[c] - bn) * (a[c] - bn);
            }
            esum[0] = 0.5 * v.ks * e;
            if (o.f) {
                for (int c = 0; c < D; ++c) {
                    o.f[((size_t)(o.P - 1) * v.d + c) * o.ldf + l] += FP[c];
                    o.f[((size_t)c) * o.ldf + l] += F1[c];
                }
            }
            if (o.g1) {
                // a device wait that gave up makes every gradient NaN
                const double gs =
                    *(volatile int*)v.err != 0 ? __longlong_as_double(0x7ff8000000000000LL) : *o.gscale;
                for (int c = 0; c < D; ++c) {
                    o.g1[(size_t)c * o.ldg + l] = -gs * F1[c];
                    o.gP[(size_t)c * o.ldg + l] = -gs * FP[c];
                }
            }
        }
    }
    block_reduce<1>(esum, red);
    if (threadIdx.x == 0 && o.part) o.part[blockIdx.x] = esum[0];
}

template <int D>
__global__ void __launch_bounds__(256) xdf_finalize_kernel(XView v, FinalizeOut o) { finalize_body<D>(v, o); }

// ------------------------------------------------------------------------
// Self-contained recursion for small systems (batched replicas): one block per
// replica and direction does every product of the solve itself, so it waits
// on no other block.  Iteration it (block J) multiplies, in chunks of at most
// XS_CHUNK tiles streamed through shared memory by bulk copies:
//   list entry 0  Q_J (forward) / P_J (backward) by the previous solution block,
//   list entry 1  G_J by h_J (every contribution to h_J is in by then),
//   list entry m  (m >= 2) M_{J-1+m, J-1} (forward) / M_{J+1, J+1-m} (backward)
//                 by the previous solution block, added into h of block
//                 J-1+m / J+1-m (right-looking update).
// Chunk 0 holds entries 0 and 1, so the dependent chain per iteration is one
// chunk's products and one reduction.  Warps 0-5 compute (work split as in
// chain_segments, with the chunk's tile count for W); warp 7 publishes.

#define XS_CHUNK 6
#define XS_SLOTS (2 * XS_CHUNK)
#define XS_NBMAX 64  // blocks of the largest replica (N <= 2047)

struct SoloS {
    float4 xv[XDF_XR][32];          // solution blocks (ring)
    float4 h[XS_NBMAX][32];         // h of every block
    float4 r[XDF_NSEG][32];         // phase-1 partials, slot 2 w + j
    int seg_m[XS_CHUNK + 1][XDF_NSEG], seg_c0[XS_CHUNK + 1][XDF_NSEG], seg_c1[XS_CHUNK + 1][XDF_NSEG];
    int red[XS_CHUNK + 1][XS_CHUNK][4], nred[XS_CHUNK + 1][XS_CHUNK];  // partial slots of each tile
    int y_ready, published, abort;
    unsigned long long mb[2];
};

template <int DIR>
__device__ __forceinline__ int solo_nband(const XView& v, int it)
{
    if (it == 0) return 0;
    const int J = chain_block<DIR>(v, it);
    return DIR == 0 ? v.nb - 1 - J : J;
}

// Global tile of list entry g of iteration it (null if absent).
template <int DIR>
__device__ __forceinline__ const XTile* solo_tile(const XView& v, int it, int g)
{
    const int J = chain_block<DIR>(v, it);
    if (g == 1) return v.G + J;
    if (it == 0) return nullptr;
    if (g == 0) return (DIR == 0 ? v.Q : v.P) + J;
    if (g - 2 >= solo_nband<DIR>(v, it)) return nullptr;
    return v.M + (DIR == 0 ? xdf_tile_index(v, J - 1 + g, J - 1) : xdf_tile_index(v, J + 1, J + 1 - g));
}

// Bulk copies of chunk ch of iteration it into ring half q & 1 (one thread).
template <int DIR>
__device__ void solo_issue(const XView& v, DfwTile* Tall, SoloS* ss, int q, int it, int ch)
{
    const int slot = q & 1, L = 2 + solo_nband<DIR>(v, it), n = min(XS_CHUNK, L - XS_CHUNK * ch);
    DfwTile* T = Tall + slot * XS_CHUNK;
    unsigned cnt = 0;
    for (int k = 0; k < n; ++k) cnt += solo_tile<DIR>(v, it, XS_CHUNK * ch + k) ? 1u : 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&ss->mb[slot], cnt * (unsigned)sizeof(XTile));
    for (int k = 0; k < n; ++k) {
        const XTile* src = solo_tile<DIR>(v, it, XS_CHUNK * ch + k);
        if (src) bulk_g2s(&T[k], src, (unsigned)sizeof(XTile), &ss->mb[slot]);
    }
}

// the chunk after (it, ch)
template <int DIR>
__device__ __forceinline__ void solo_advance(const XView& v, int& it, int& ch)
{
    if (++ch * XS_CHUNK >= 2 + solo_nband<DIR>(v, it)) {
        ch = 0;
        ++it;
    }
}

template <int DIR>
__device__ void xsolo(const XView& v, DfwTile* Tall, SoloS* ss)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nb = v.nb;
    const int lim = v.spin_limit;
    if (tid == 0) {
        ss->y_ready = -1;
        ss->published = -1;
        ss->abort = 0;
        for (int n = 1; n <= XS_CHUNK; ++n) {
            chain_segments(n, ss->seg_m[n], ss->seg_c0[n], ss->seg_c1[n]);
            for (int k = 0; k < XS_CHUNK; ++k) {
                int c = 0;
                for (int s = 0; s < XDF_NSEG; ++s)
                    if (ss->seg_m[n][s] == k && c < 4) ss->red[n][k][c++] = s;
                ss->nred[n][k] = c;
            }
        }
        mbar_init(&ss->mb[0], 1);
        mbar_init(&ss->mb[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int i = tid; i < nb * 32; i += blockDim.x) ss->h[i >> 5][i & 31] = dfw_pack(dfw_zero());
    block_sync();

    if (w == XDF_WARPS - 1) {
        // ---- publisher: solution blocks and weight products to global memory
        for (int it = 0; it < nb; ++it) {
            if (!smem_wait_ge(&ss->y_ready, it, &ss->abort, lim, v.err, 0x620000 + it)) break;
            const int J = chain_block<DIR>(v, it), n = 32 * J + lane;
            const dfw xw = dfw_unpack(ss->xv[it % XDF_XR][lane]);
            const df xm = df{xw.h, xw.l};
            (DIR == 0 ? v.yh : v.ch)[n] = xm.h;
            (DIR == 0 ? v.yl : v.cl)[n] = xm.l;
            (DIR == 0 ? v.ye : v.ce)[n] = xw.e;
            for (int c = 0; c < v.d; ++c) {
                df e = df{0.f, 0.f};
                if (DIR == 0) e = df{v.bh[(size_t)c * v.npad + n], v.bl[(size_t)c * v.npad + n]};
                else if (n >= 1 && n <= v.N) e = df{v.ah[(size_t)c * v.npad + n - 1], v.al[(size_t)c * v.npad + n - 1]};
                const df u = df_mul(xm, e);
                (DIR == 0 ? v.uh : v.wh)[(size_t)c * v.npad + n] = u.h;
                (DIR == 0 ? v.ul : v.wl)[(size_t)c * v.npad + n] = u.l;
            }
            __syncwarp();
            if (lane == 0) vstore(&ss->published, it);
            __syncwarp();
        }
        return;
    }
    if (w == XDF_WARPS - 2) return;

    // ---- compute warps 0-5 (never leave the loop early; see xchain)
    int qi = 0, ich = 0, q_issued = -1;  // warp 5 lane 0: next chunk to issue
    if (w == 5 && lane == 0) {
        for (int k = 0; k < 2 && qi < nb; ++k) {
            solo_issue<DIR>(v, Tall, ss, k, qi, ich);
            q_issued = k;
            solo_advance<DIR>(v, qi, ich);
        }
    }
    int q = 0;
    for (int it = 0; it < nb; ++it) {
        const int J = chain_block<DIR>(v, it), L = 2 + solo_nband<DIR>(v, it);
        const int xp = (it + XDF_XR - 1) % XDF_XR;
        for (int ch = 0; ch * XS_CHUNK < L; ++ch, ++q) {
            const int slot = q & 1, n = min(XS_CHUNK, L - XS_CHUNK * ch);
            DfwTile* T = Tall + slot * XS_CHUNK;
            mbar_wait(&ss->mb[slot], (unsigned)(q >> 1), lim, v.err, &ss->abort, 0x630000 + it, false);
            // phase 1
            dfw x0 = dfw_zero();
            if (it == 0 && w == 0) x0 = DIR == 0 ? tile_get(&T[1], lane, 0) : tile_get(&T[1], v.N - 32 * J, lane);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = ss->seg_m[n][2 * w + j];
                if (k < 0) continue;
                const int g = XS_CHUNK * ch + k;
                dfw p = dfw_zero();
                if (it >= 1 && solo_tile<DIR>(v, it, g)) {
                    const float4* xv = g == 1 ? ss->h[J] : ss->xv[xp];
                    const int c0 = ss->seg_c0[n][2 * w + j], c1 = ss->seg_c1[n][2 * w + j];
                    p = DIR == 0 ? dot_seg<false>(&T[k], lane, xv, c0, c1) : dot_seg<true>(&T[k], lane, xv, c0, c1);
                }
                ss->r[2 * w + j][lane] = dfw_pack(p);
            }
            compute_sync();
            // phase 2: reductions
            if (ch == 0 && w == 0) {
                smem_wait_ge(&ss->published, it - XDF_XR, &ss->abort, lim, v.err, 0x640000 + it);
                dfw x = x0;
                if (it >= 1) {
                    dfw t[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) t[i] = dfw_zero();
                    int c = 0;
                    for (int k = 0; k < 2; ++k)
                        for (int i = 0; i < ss->nred[n][k]; ++i) {
                            const dfw pv = dfw_unpack(ss->r[ss->red[n][k][i]][lane]);
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (u == c) t[u] = pv;
                            ++c;
                        }
                    x = dfw_sum8(t, c);
                }
                ss->xv[it % XDF_XR][lane] = dfw_pack(x);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) vstore(&ss->y_ready, it);
                __syncwarp();
            }
            // band tile k of this chunk: reducer warp k - 1 in chunk 0, k otherwise
            for (int k = (ch == 0 ? 2 : 0); k < n; ++k) {
                if (w != (ch == 0 ? k - 1 : k)) continue;
                const int g = XS_CHUNK * ch + k;
                if (!solo_tile<DIR>(v, it, g)) continue;
                const int tgt = DIR == 0 ? J - 1 + g : J + 1 - g;
                dfw t[8];
                t[0] = dfw_unpack(ss->h[tgt][lane]);
#pragma unroll
                for (int i = 0; i < 4; ++i) t[1 + i] = i < ss->nred[n][k] ? dfw_unpack(ss->r[ss->red[n][k][i < 4 ? i : 0]][lane]) : dfw_zero();
                t[5] = t[6] = t[7] = dfw_zero();
                ss->h[tgt][lane] = dfw_pack(dfw_sum8(t, 1 + ss->nred[n][k]));
            }
            if (w == 5 && lane == 0 && qi < nb && !vload(&ss->abort)) {
                solo_issue<DIR>(v, Tall, ss, q + 2, qi, ich);
                q_issued = q + 2;
                solo_advance<DIR>(v, qi, ich);
            }
            compute_sync();
        }
    }
    // every issued bulk copy lands before the block's shared memory is released
    if (w == 5 && lane == 0)
        for (int sl = 0; sl < 2 && sl <= q_issued; ++sl) {
            const int last = sl + ((q_issued - sl) / 2) * 2;
            mbar_wait(&ss->mb[sl], (unsigned)(last >> 1), lim, v.err, &ss->abort, 0x658000 + sl, true);
        }
}

__global__ void __launch_bounds__(XDF_THREADS, 1) xsolo_batch(const RepArgs* ra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfwTile* T = reinterpret_cast<DfwTile*>(smem_raw);
    SoloS* ss = reinterpret_cast<SoloS*>(smem_raw + XS_SLOTS * sizeof(DfwTile));
    const XView& v = ra[blockIdx.y].xv;
    if (v.xi_zero) return;
    if (blockIdx.x == 0) xsolo<0>(v, T, ss);
    else xsolo<1>(v, T, ss);
}

__global__ void __launch_bounds__(256) prep_batch(const RepArgs* ra)
{
    prep_body(ra[blockIdx.z].xv, blockIdx.x, gridDim.x);
}


// Factor tiles of every replica from a flat list of (replica, tile) pairs, grid-stride.
template <int D>
__global__ void __launch_bounds__(256) table_flat(const RepArgs* ra, const int2* list, int n)
{
    __shared__ float2 tab[256];
    __shared__ TableStage st;
    load_tab_smem(tab, ra[0].xv.tab);  // one exp table for the whole batch
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int2 e = list[i];
        table_tile_t<D>(ra[e.x].xv, e.y, tab, st);
    }
}

// Block operators of every replica over a flat list of (replica, diagonal
// block) pairs: G_J in 8-column parts (grid (4, n)), then Q_J and P_J in row
// quarters (grid (8, n)).
__global__ void __launch_bounds__(256) gparts_flat(const RepArgs* ra, const int2* list)
{
    __shared__ __align__(16) unsigned char sm[sizeof(DfwTile)];
    const int2 e = list[blockIdx.y];
    blockops_g_item(ra[e.x].xv, e.y, blockIdx.x, sm);
}

__global__ void __launch_bounds__(256) prods_flat(const RepArgs* ra, const int2* list)
{
    __shared__ __align__(16) unsigned char sm[2 * sizeof(DfwTile)];
    const int2 e = list[blockIdx.y];
    blockops_prod_item(ra[e.x].xv, e.y, blockIdx.x >> 2, blockIdx.x & 3, sm);
}


__global__ void __launch_bounds__(256) band_batch(const RepArgs* ra)
{
    const XView& v = ra[blockIdx.z].xv;
    if (v.xi_zero) return;
    band_body(v, blockIdx.x, blockIdx.y, -1);
}

__global__ void __launch_bounds__(256) finalize_batch(const RepArgs* ra)
{
    const RepArgs& a = ra[blockIdx.z];
    if (a.xv.d == 1) finalize_body<1>(a.xv, a.fo);
    else if (a.xv.d == 2) finalize_body<2>(a.xv, a.fo);
    else finalize_body<3>(a.xv, a.fo);
}

// The recursion and band sums of the batched exchange step as one persistent
// launch (work list in pimd_batch.cuh): recursion items (the self-contained
// solve of one replica and direction, xsolo) longest first, then band items,
// each waiting until both recursions of its replica are done.
__global__ void __launch_bounds__(XDF_THREADS, 2) batch_exch_persistent(const RepArgs* ra, BatchSched sc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_ok;
    const int tid = threadIdx.x;
    for (;;) {
        block_sync();  // every thread has read the previous item's s_item and s_ok
        if (tid == 0) s_item = atomicAdd(sc.next, 1);
        block_sync();
        const int i = s_item;
        if (i >= sc.n_items) return;
        const BatchItem it = sc.items[i];
        const XView& v = ra[it.r].xv;
        if (tid == 0) {
            int ok = 1;
            if (it.type == BI_BAND)
                ok = wait_flag(&sc.done[it.r * 4 + BI_REC], sc.need[it.r * 4 + BI_REC], sc.err, sc.spin_limit,
                               0x900000 + (it.r & 0xFFFF));
            s_ok = ok;
        }
        block_sync();
        if (s_ok) {
            if (it.type == BI_REC) {
                DfwTile* T = reinterpret_cast<DfwTile*>(smem_raw);
                SoloS* ss = reinterpret_cast<SoloS*>(smem_raw + XS_SLOTS * sizeof(DfwTile));
                if (it.a == 0) xsolo<0>(v, T, ss);
                else xsolo<1>(v, T, ss);
            } else {
                band_body(v, it.a, it.b, -1);
            }
        }
        block_sync();
        if (tid == 0 && it.type != BI_BAND) {
            __threadfence();
            atomicAdd(&sc.done[it.r * 4 + it.type], 1);
        }
    }
}

// V_ends = V_xi - sum E_int = (sum_l g(l, l+1) - ln W_N)/beta with
// ln W_N = N ln xi + ln y[N] (xi = 0: the diagonal chain), from the prep
// partial sums and the forward solution (Sec. III).
// A device wait that gave up during the call (error word set) gives NaN.
__global__ void xdf_vb_value_kernel(XView v, int nprep, double* V_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (*(volatile int*)v.err != 0) {
        *V_out = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    double gl = 0.0, l0 = 0.0;
    for (int i = 0; i < nprep; ++i) {
        gl += v.lsum[2 * i];
        l0 += v.lsum[2 * i + 1];
    }
    const double lam = v.xi_zero ? l0 : v.N * v.log_xi + dfw_log_df(xget(v.yh, v.yl, v.ye, v.N), v.tab);
    *V_out = (gl - lam) / v.beta;
}

// ------------------------------------------------------------------------
// Latency probe of the recursion chain: the dependent core of one block
// iteration, y_it = Q_k y_{it-1} + G_k s with k = it mod nblk (the chain's
// y_J = Q_J y_{J-1} + G_J s_J).  The Q and G tiles sit in shared memory as
// wide-exponent double-float tiles; the two products are split over
// 2*split warps exactly as the chain's phase 1 splits them (split warps per
// tile, 32/split columns each, compensated segment dots), warp 0 sums the
// partials into the new solution block (phase 2), and two named barriers
// close each iteration.  No global memory, helper partials, tile copies or
// publication: what is left is the work every block of the chain has to do
// in sequence, so nb times its cycle count is a floor under the chain.
__global__ void __launch_bounds__(XDF_THREADS, 1)
    xdf_probe_chain_kernel(const double* Q, const double* G, const double* y0, const double* sv, int nblk, int n_iter,
                           int split, double* y_out, long long* cycles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfwTile* TQ = reinterpret_cast<DfwTile*>(smem_raw);
    DfwTile* TG = TQ + nblk;
    __shared__ float4 xv[2][32];
    __shared__ float4 sx[32];
    __shared__ float4 rp[XDF_WARPS][32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int q = tid; q < nblk * 1024; q += blockDim.x) {
        const int k = q >> 10, rr = (q >> 5) & 31, cc = q & 31;
        tile_put(&TQ[k], rr, cc, dfw_norm(df_from_double(Q[q]), 0));
        tile_put(&TG[k], rr, cc, dfw_norm(df_from_double(G[q]), 0));
    }
    if (tid < 32) {
        xv[0][tid] = dfw_pack(dfw_norm(df_from_double(y0[tid]), 0));
        sx[tid] = dfw_pack(dfw_norm(df_from_double(sv[tid]), 0));
    }
    block_sync();
    const int nw = 2 * split, cw = 32 / split;
    const long long t0 = clock64();
    if (w < nw) {
        const bool isq = w < split;
        const int c0 = (isq ? w : w - split) * cw;
        for (int it = 0; it < n_iter; ++it) {
            const int k = it % nblk;
            const dfw p = isq ? dot_seg<false>(&TQ[k], lane, xv[it & 1], c0, c0 + cw)
                              : dot_seg<false>(&TG[k], lane, sx, c0, c0 + cw);
            rp[w][lane] = dfw_pack(p);
            __syncwarp();
            asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");
            if (w == 0) {
                dfw t[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) t[i] = i < nw ? dfw_unpack(rp[i][lane]) : dfw_zero();
                xv[(it + 1) & 1][lane] = dfw_pack(dfw_sum8(t, nw));
            }
            __syncwarp();
            asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");
        }
    }
    const long long t1 = clock64();
    block_sync();
    if (tid == 0) *cycles = t1 - t0;
    if (tid < 32) y_out[tid] = dfw_to_double(dfw_unpack(xv[n_iter & 1][tid]));
}

}  // namespace

cudaError_t xdf_launch_probe_chain(const double* Q, const double* G, const double* y0, const double* s, int nblk,
                                   int n_iter, int split, double* y_out, long long* cycles, cudaStream_t st)
{
    if (nblk < 1 || nblk > 8 || n_iter < 1 || (split != 1 && split != 2 && split != 4)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * nblk * sizeof(DfwTile);
    static DeviceOnce attr_once;
    cudaError_t e = device_once(attr_once, [] {
        return cudaFuncSetAttribute(xdf_probe_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(16 * sizeof(DfwTile)));
    });
    if (e != cudaSuccess) return e;
    xdf_probe_chain_kernel<<<1, XDF_THREADS, smem, st>>>(Q, G, y0, s, nblk, n_iter, split, y_out, cycles);
    return cudaGetLastError();
}

// prep and finalize do FP64 work per particle: 64-thread blocks spread it over more SMs
constexpr int XDF_SMALL_T = 64;
int xdf_prep_blocks(int npad) { return min(152 * 4, (npad + XDF_SMALL_T - 1) / XDF_SMALL_T); }
constexpr int XDF_FIN_T = 64;  // finalize: one thread per particle
int xdf_finalize_blocks(int N) { return (N + XDF_FIN_T - 1) / XDF_FIN_T; }

size_t xdf_recursion_smem(int W)
{
    (void)W;
    const size_t tab_off = (XDF_TILES * sizeof(DfwTile) + XDF_WSLOTS * sizeof(WeightSmem) + sizeof(ChainS) + 15) & ~(size_t)15;
    return tab_off + 256 * sizeof(float2);
}

static size_t band_smem(int nw) { return nw * (sizeof(DfwTile) + sizeof(WeightSmem) + 32 * sizeof(DVAcc)); }

cudaError_t xdf_launch_forward(const XView& v, cudaStream_t st, ProfMarks* pm, const ForceWork* fw, int n_force)
{
    xdf_prep_kernel<<<xdf_prep_blocks(v.npad), XDF_SMALL_T, 0, st>>>(v);
    prof_mark(pm, "exch_prep", st);
    if (v.xi_zero) return cudaGetLastError();
    const long long nt = xdf_ntiles(v.nb, v.W, v.store);
    const int tgrid = (int)min(nt, (long long)152 * 16);
    xdf_table_kernel<<<tgrid, 256, 0, st>>>(v, nt);
    prof_mark(pm, "exch_table", st);
    static DeviceOnce attr_once;
    cudaError_t e = device_once(attr_once, [] {
        return cudaFuncSetAttribute(xdf_recursion_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)xdf_recursion_smem(XDF_MAXW));
    });
    if (e != cudaSuccess) return e;
    // block operators: G_J in 8-column parts, then the row quarters of Q_J and P_J
    xdf_gparts_kernel<<<dim3(4, v.nb), 256, 0, st>>>(v);
    prof_mark(pm, "exch_gparts", st);
    xdf_prods_kernel<<<dim3(8, v.nb), 256, 0, st>>>(v);
    prof_mark(pm, "exch_prods", st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the helper and force-worker blocks form the band sums at their end
    if (band_smem(8) > xdf_recursion_smem(v.W) || v.n_help_f + v.n_help_b < 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    ForceWork none;
    memset(&none, 0, sizeof none);
    if (!fw || n_force < 0) n_force = 0;
    cfg.gridDim = dim3(2 + v.n_help_f + v.n_help_b + n_force);
    cfg.blockDim = dim3(XDF_THREADS);
    cfg.dynamicSmemBytes = xdf_recursion_smem(v.W);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, xdf_recursion_kernel, v, n_force > 0 ? *fw : none);
    prof_mark(pm, "exch_recursion", st);
    return e;
}

cudaError_t xdf_launch_adjoint(const XView& v, const FinalizeOut& o, cudaStream_t st, ProfMarks* pm)
{
    // the band sums were formed inside the recursion launch (band_worker)
    if (v.d == 1) xdf_finalize_kernel<1><<<xdf_finalize_blocks(v.N), XDF_FIN_T, 0, st>>>(v, o);
    else if (v.d == 2) xdf_finalize_kernel<2><<<xdf_finalize_blocks(v.N), XDF_FIN_T, 0, st>>>(v, o);
    else xdf_finalize_kernel<3><<<xdf_finalize_blocks(v.N), XDF_FIN_T, 0, st>>>(v, o);
    prof_mark(pm, "exch_finalize", st);
    return cudaGetLastError();
}

static __global__ void xdf_lntab_kernel(double* lnn, int n)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) lnn[q] = q >= 1 ? log((double)q) : 0.0;
}

// ln n for n < npad (entry 0 is 0), once per workspace: the row constants
// need ln n every step.
cudaError_t xdf_fill_lntab(double* dev_lnn, int npad, cudaStream_t st)
{
    if (npad < 1) return cudaSuccess;
    xdf_lntab_kernel<<<(npad + 255) / 256, 256, 0, st>>>(dev_lnn, npad);
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

size_t xsolo_smem() { return XS_SLOTS * sizeof(DfwTile) + sizeof(SoloS); }

cudaError_t batch_launch_exchange(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm)
{
    static DeviceOnce attr_once;
    cudaError_t e = device_once(attr_once, [] {
        cudaError_t r = cudaFuncSetAttribute(xsolo_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsolo_smem());
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(band_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem(8));
        return r;
    });
    if (e != cudaSuccess) return e;
    prep_batch<<<dim3(g.gx_prep, 1, g.R), XDF_SMALL_T, 0, st>>>(ra);
    prof_mark(pm, "batch_exch_prep", st);
    e = batch_launch_tables_ops(ra, g, st, pm);
    if (e != cudaSuccess) return e;
    xsolo_batch<<<dim3(2, g.R), XDF_THREADS, xsolo_smem(), st>>>(ra);
    prof_mark(pm, "batch_exch_recursion", st);
    band_batch<<<dim3(g.nb_max, 2, g.R), 256, band_smem(8), st>>>(ra);
    prof_mark(pm, "batch_exch_band", st);
    finalize_batch<<<dim3(g.gx_fin, 1, g.R), XDF_FIN_T, 0, st>>>(ra);
    prof_mark(pm, "batch_exch_finalize", st);
    return cudaGetLastError();
}

static size_t persistent_smem() { return std::max(xsolo_smem(), band_smem(8)); }

cudaError_t batch_launch_exchange_persistent(const RepArgs* ra, const BatchSched& sc, int blocks, cudaStream_t st)
{
    static DeviceOnce attr_once;
    cudaError_t e = device_once(attr_once, [] {
        return cudaFuncSetAttribute(batch_exch_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)persistent_smem());
    });
    if (e != cudaSuccess) return e;
    batch_exch_persistent<<<blocks, XDF_THREADS, persistent_smem(), st>>>(ra, sc);
    return cudaGetLastError();
}

// prep, factor tiles and block operators of every replica (flat lists, no idle blocks)
cudaError_t batch_launch_prep_tables_ops(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm)
{
    prep_batch<<<dim3(g.gx_prep, 1, g.R), XDF_SMALL_T, 0, st>>>(ra);
    prof_mark(pm, "batch_exch_prep", st);
    cudaError_t e = batch_launch_tables_ops(ra, g, st, pm);
    return e;
}

cudaError_t batch_launch_tables_ops(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm)
{
    if (g.n_tiles > 0) {
        const int grid = std::min(g.n_tiles, 152 * 8);
        if (g.d == 1) table_flat<1><<<grid, 256, 0, st>>>(ra, g.tiles, g.n_tiles);
        else if (g.d == 2) table_flat<2><<<grid, 256, 0, st>>>(ra, g.tiles, g.n_tiles);
        else table_flat<3><<<grid, 256, 0, st>>>(ra, g.tiles, g.n_tiles);
    }
    prof_mark(pm, "batch_exch_table", st);
    if (g.n_blocks > 0) {
        gparts_flat<<<dim3(4, g.n_blocks), 256, 0, st>>>(ra, g.blocks);
        prods_flat<<<dim3(8, g.n_blocks), 256, 0, st>>>(ra, g.blocks);
    }
    prof_mark(pm, "batch_exch_blockops", st);
    return cudaGetLastError();
}

cudaError_t batch_launch_finalize(const RepArgs* ra, const BatchGrid& g, cudaStream_t st)
{
    finalize_batch<<<dim3(g.gx_fin, 1, g.R), XDF_FIN_T, 0, st>>>(ra);
    return cudaGetLastError();
}

cudaError_t xdf_launch_vb_value(const XView& v, double* V_out, cudaStream_t st)
{
    xdf_vb_value_kernel<<<1, 32, 0, st>>>(v, xdf_prep_blocks(v.npad), V_out);
    return cudaGetLastError();
}
