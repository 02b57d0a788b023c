// Double-float exchange kernels (arXiv 2404.02628, Sec. III): prep, factor
// table, block operators, look-ahead recursion, band sums, endpoint forces.
// The equations are stated in pimd_xdf.cuh.
#include <math.h>
#include <stdio.h>

#include "pimd_xdf.cuh"

namespace {

struct DfwTile {  // 32x32 dfw matrix in shared memory, padded rows
    float h[32 * XDF_LD];
    float l[32 * XDF_LD];
    int e[32 * XDF_LD];
};

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

// Copy a global 32x32 dfw tile (row-major, 1024 entries) into shared memory.
__device__ __forceinline__ void stage_block(DfwTile* s, const float* h, const float* l, const int* e)
{
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
        const int r = q >> 5, c = q & 31;
        s->h[r * XDF_LD + c] = h[q];
        s->l[r * XDF_LD + c] = l[q];
        s->e[r * XDF_LD + c] = e[q];
    }
}

__device__ __forceinline__ void stage_warp(DfwTile* s, const float* h, const float* l, const int* e, int lane)
{
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
        s->h[r * XDF_LD + lane] = h[r * 32 + lane];
        s->l[r * XDF_LD + lane] = l[r * 32 + lane];
        s->e[r * XDF_LD + lane] = e[r * 32 + lane];
    }
}

__device__ __forceinline__ dfw tile_get(const DfwTile* s, int r, int c)
{
    const int q = r * XDF_LD + c;
    return dfw{s->h[q], s->l[q], s->e[q]};
}

// sum_{t in [t0,t1)} A[r][t] * x[t]  (x given as per-t dfw in shared arrays)
__device__ __forceinline__ dfw dot_row_vec(const DfwTile* A, int r, const float* xh, const float* xl, const int* xe,
                                           int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[r * XDF_LD + t] + xe[t]);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int q = r * XDF_LD + t;
        const float f = pow2f(A->e[q] + xe[t] - E);
        s = df_add(s, df_scale(df_mul(df{A->h[q], A->l[q]}, df{xh[t], xl[t]}), f));
    }
    return dfw_norm(s, E);
}

// sum_{t in [t0,t1)} A[t][c] * x[t]  (transposed)
__device__ __forceinline__ dfw dot_col_vec(const DfwTile* A, int c, const float* xh, const float* xl, const int* xe,
                                           int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[t * XDF_LD + c] + xe[t]);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int q = t * XDF_LD + c;
        const float f = pow2f(A->e[q] + xe[t] - E);
        s = df_add(s, df_scale(df_mul(df{A->h[q], A->l[q]}, df{xh[t], xl[t]}), f));
    }
    return dfw_norm(s, E);
}

// (A B)[r][c] over t in [t0, t1)
__device__ __forceinline__ dfw dot_mat(const DfwTile* A, const DfwTile* B, int r, int c, int t0, int t1)
{
    int E = WEF_ZERO_E;
    for (int t = t0; t < t1; ++t) E = max(E, A->e[r * XDF_LD + t] + B->e[t * XDF_LD + c]);
    if (E <= WEF_ZERO_E / 2) return dfw_zero();
    df s = df{0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const int qa = r * XDF_LD + t, qb = t * XDF_LD + c;
        const float f = pow2f(A->e[qa] + B->e[qb] - E);
        s = df_add(s, df_scale(df_mul(df{A->h[qa], A->l[qa]}, df{B->h[qb], B->l[qb]}), f));
    }
    return dfw_norm(s, E);
}

// Weighted row sums of tile A for row r: s = sum_t A[r][t] w[t], v = sum_t A[r][t] w[t] u_c[t]
// where wu[c][t] = w[t].mant * u_c[t] (relative to w's exponent).
struct WeightSmem {
    float wh[32], wl[32];
    int we[32];
    float uh[3][32], ul[3][32];
};

__device__ __forceinline__ DVAcc weighted_rows(const DfwTile* A, const WeightSmem* w, int r, int d)
{
    DVAcc out = dv_zero();
    int E = WEF_ZERO_E;
    for (int t = 0; t < 32; ++t) E = max(E, A->e[r * XDF_LD + t] + w->we[t]);
    if (E <= WEF_ZERO_E / 2) return out;
    for (int t = 0; t < 32; ++t) {
        const int q = r * XDF_LD + t;
        const float f = pow2f(A->e[q] + w->we[t] - E);
        const df a = df_scale(df{A->h[q], A->l[q]}, f);
        out.s = df_add(out.s, df_mul(a, df{w->wh[t], w->wl[t]}));
        for (int c = 0; c < d; ++c) out.v[c] = df_add(out.v[c], df_mul(a, df{w->uh[c][t], w->ul[c][t]}));
    }
    out.e = E;
    dv_renorm(out);
    return out;
}

__device__ __forceinline__ DVAcc weighted_cols(const DfwTile* A, const WeightSmem* w, int c0, int d)
{
    DVAcc out = dv_zero();
    int E = WEF_ZERO_E;
    for (int t = 0; t < 32; ++t) E = max(E, A->e[t * XDF_LD + c0] + w->we[t]);
    if (E <= WEF_ZERO_E / 2) return out;
    for (int t = 0; t < 32; ++t) {
        const int q = t * XDF_LD + c0;
        const float f = pow2f(A->e[q] + w->we[t] - E);
        const df a = df_scale(df{A->h[q], A->l[q]}, f);
        out.s = df_add(out.s, df_mul(a, df{w->wh[t], w->wl[t]}));
        for (int c = 0; c < d; ++c) out.v[c] = df_add(out.v[c], df_mul(a, df{w->uh[c][t], w->ul[c][t]}));
    }
    out.e = E;
    dv_renorm(out);
    return out;
}

// Forward weights of column block I: y[k] and y[k] b_k.
__device__ __forceinline__ void load_wf(const XView& v, WeightSmem* w, int I, int lane)
{
    const int k = 32 * I + lane;
    const float h = __ldcg(&v.yh[k]), l = __ldcg(&v.yl[k]);
    const int e = __ldcg(&v.ye[k]);
    w->wh[lane] = h;
    w->wl[lane] = l;
    w->we[lane] = e;
    for (int c = 0; c < 3; ++c) {
        df u = df{0.f, 0.f};
        if (c < v.d && k < v.N) u = df_mul(df{h, l}, df{v.bh[(size_t)c * v.npad + k], v.bl[(size_t)c * v.npad + k]});
        w->uh[c][lane] = u.h;
        w->ul[c][lane] = u.l;
    }
}

// Backward weights of row block J: c[n] and c[n] a_{n-1}.
__device__ __forceinline__ void load_wb(const XView& v, WeightSmem* w, int J, int lane)
{
    const int n = 32 * J + lane;
    const float h = __ldcg(&v.ch[n]), l = __ldcg(&v.cl[n]);
    const int e = __ldcg(&v.ce[n]);
    w->wh[lane] = h;
    w->wl[lane] = l;
    w->we[lane] = e;
    for (int c = 0; c < 3; ++c) {
        df u = df{0.f, 0.f};
        if (c < v.d && n >= 1 && n <= v.N)
            u = df_mul(df{h, l}, df{v.ah[(size_t)c * v.npad + n - 1], v.al[(size_t)c * v.npad + n - 1]});
        w->uh[c][lane] = u.h;
        w->ul[c][lane] = u.l;
    }
}

// Tile (J,I) of M into shared memory: stored tiles are copied, others computed.
__device__ __forceinline__ void get_tile_warp(const XView& v, DfwTile* s, int J, int I, int lane, const float2* tab)
{
    if (v.store || J - I < v.W) {
        const long long t = xdf_tile_index(v, J, I);
        stage_warp(s, v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024, lane);
        return;
    }
    for (int r = 0; r < 32; ++r) {
        const dfw m = xM(v, 32 * J + r, 32 * I + lane, tab);
        s->h[r * XDF_LD + lane] = m.h;
        s->l[r * XDF_LD + lane] = m.l;
        s->e[r * XDF_LD + lane] = m.e;
    }
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
    __syncthreads();
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int J, I;
        if (v.store) {
            J = (int)floor((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
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
            dfw m = dfw_zero();
            if (I >= 0) m = xM(v, 32 * J + (q >> 5), 32 * I + (q & 31), tab);
            Mh[q] = m.h;
            Ml[q] = m.l;
            Me[q] = m.e;
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
        stage_block(L, v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024);
        if (J >= 1) {
            const long long ts = xdf_tile_index(v, J, J - 1);
            stage_block(Ms, v.Mh + ts * 1024, v.Ml + ts * 1024, v.Me + ts * 1024);
        }
        if (J + 1 < v.nb) {
            const long long tp = xdf_tile_index(v, J + 1, J);
            stage_block(Mp, v.Mh + tp * 1024, v.Ml + tp * 1024, v.Me + tp * 1024);
        }
    }
    __syncthreads();
    if (w == 0) {
        // row by row: G[r][c] = delta_rc + sum_{t=c}^{r-1} L[r][t] G[t][c]
        for (int r = 0; r < 32; ++r) {
            dfw g;
            if (lane < r) {
                int E = WEF_ZERO_E;
                for (int t = lane; t < r; ++t) E = max(E, L->e[r * XDF_LD + t] + G->e[t * XDF_LD + lane]);
                if (E <= WEF_ZERO_E / 2) {
                    g = dfw_zero();
                } else {
                    df s = df{0.f, 0.f};
                    for (int t = lane; t < r; ++t) {
                        const int qa = r * XDF_LD + t, qb = t * XDF_LD + lane;
                        const float f = pow2f(L->e[qa] + G->e[qb] - E);
                        s = df_add(s, df_scale(df_mul(df{L->h[qa], L->l[qa]}, df{G->h[qb], G->l[qb]}), f));
                    }
                    g = dfw_norm(s, E);
                }
            } else if (lane == r) {
                g = dfw{1.f, 0.f, 0};
            } else {
                g = dfw_zero();
            }
            G->h[r * XDF_LD + lane] = g.h;
            G->l[r * XDF_LD + lane] = g.l;
            G->e[r * XDF_LD + lane] = g.e;
            __syncwarp();
        }
    }
    __syncthreads();
    const size_t base = (size_t)J * 1024;
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
        const int r = q >> 5, c = q & 31;
        v.Gh[base + q] = G->h[r * XDF_LD + c];
        v.Gl[base + q] = G->l[r * XDF_LD + c];
        v.Ge[base + q] = G->e[r * XDF_LD + c];
        dfw Q = dfw_zero(), Pm = dfw_zero();
        if (J >= 1) Q = dot_mat(G, Ms, r, c, 0, r + 1);
        if (J + 1 < v.nb) Pm = dot_mat(Mp, G, r, c, c, 32);
        v.Qh[base + q] = Q.h;
        v.Ql[base + q] = Q.l;
        v.Qe[base + q] = Q.e;
        v.Ph[base + q] = Pm.h;
        v.Pl[base + q] = Pm.l;
        v.Pe[base + q] = Pm.e;
    }
}

// ------------------------------------------------------------------------
// recursion: chain blocks and helpers

struct ChainS {
    float xh[32], xl[32];     // current solution block
    int xe[32];
    float pvh[32], pvl[32];   // previous solution block
    int pve[32];
    float ghh[32], ghl[32];   // G h for the next block
    int ghe[32];
    float hh[XDF_MAXW][32], hl[XDF_MAXW][32];  // band accumulators (ring)
    int he[XDF_MAXW][32];
    float rh[XDF_WARPS][32], rl[XDF_WARPS][32];  // cross-warp partials
    int re[XDF_WARPS][32];
    float tmph[32], tmpl[32];
    int tmpe[32];
    DVAcc hm[XDF_WARPS][32];  // helper merge
    int abort;
};

__device__ __forceinline__ dfw chain_get(const float* h, const float* l, const int* e, int i) { return dfw{h[i], l[i], e[i]}; }
__device__ __forceinline__ void chain_put(float* h, float* l, int* e, int i, dfw x)
{
    h[i] = x.h;
    l[i] = x.l;
    e[i] = x.e;
}

// Forward chain block.  Shared tiles: T[0] = Q_J, T[1] = G_{J+1}, T[2..W-1] = M_{J+m,J}.
__device__ void xchain_forward(const XView& v, DfwTile* T, ChainS* cs)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int* flag_chain = v.flags;
    const int* flag_part = v.flags + 2 * v.nb;
    const int W = v.W;
    if (tid == 0) cs->abort = 0;
    for (int m = 0; m < W; ++m)
        if (tid < 32) chain_put(cs->hh[m], cs->hl[m], cs->he[m], tid, dfw_zero());
    for (int J = 0; J < v.nb; ++J) {
        // stage the operators and band tiles of this iteration
        if (J >= 1) stage_block(&T[0], v.Qh + (size_t)J * 1024, v.Ql + (size_t)J * 1024, v.Qe + (size_t)J * 1024);
        else stage_block(&T[0], v.Gh, v.Gl, v.Ge);  // J = 0: y_0 = G_0 e_0
        if (J + 1 < v.nb)
            stage_block(&T[1], v.Gh + (size_t)(J + 1) * 1024, v.Gl + (size_t)(J + 1) * 1024, v.Ge + (size_t)(J + 1) * 1024);
        for (int m = 2; m < W; ++m)
            if (J + m < v.nb) {
                const long long t = xdf_tile_index(v, J + m, J);
                stage_block(&T[m], v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024);
            }
        __syncthreads();
        // critical: y_J = GH_J + Q_J y_{J-1}
        if (J == 0) {
            if (w == 0) chain_put(cs->xh, cs->xl, cs->xe, lane, tile_get(&T[0], lane, 0));
        } else {
            const dfw p = dot_row_vec(&T[0], lane, cs->pvh, cs->pvl, cs->pve, 4 * w, 4 * w + 4);
            chain_put(cs->rh[w], cs->rl[w], cs->re[w], lane, p);
            __syncthreads();
            if (w == 0) {
                dfw s = chain_get(cs->ghh, cs->ghl, cs->ghe, lane);
                for (int q = 0; q < XDF_WARPS; ++q) s = dfw_add(s, chain_get(cs->rh[q], cs->rl[q], cs->re[q], lane));
                chain_put(cs->xh, cs->xl, cs->xe, lane, s);
            }
        }
        if (w == 0) {
            const int n = 32 * J + lane;
            v.yh[n] = cs->xh[lane];
            v.yl[n] = cs->xl[lane];
            v.ye[n] = cs->xe[lane];
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release(&flag_chain[J], 1);
        }
        __syncthreads();
        // band: h_{J+m} += M_{J+m,J} y_J   (warp m-2 handles band tile m)
        if (w >= 0 && w + 2 < W && J + w + 2 < v.nb) {
            const int m = w + 2;
            const dfw p = dot_row_vec(&T[m], lane, cs->xh, cs->xl, cs->xe, 0, 32);
            const int slot = (J + m) % W;
            chain_put(cs->hh[slot], cs->hl[slot], cs->he[slot], lane,
                      dfw_add(chain_get(cs->hh[slot], cs->hl[slot], cs->he[slot], lane), p));
        }
        // next block's G h: warp 7 merges helper partials into h_{J+1} and applies G_{J+1}
        if (w == XDF_WARPS - 1 && J + 1 < v.nb) {
            const int Jn = J + 1, slot = Jn % W;
            dfw h = chain_get(cs->hh[slot], cs->hl[slot], cs->he[slot], lane);
            const int ns = min(v.S, Jn - W + 1);
            for (int s = 0; s < ns; ++s) {
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_part[Jn * v.S + s], 1, v.err, v.spin_limit, 0x510000 + Jn);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                const size_t idx = xpart_index(v, 0, Jn, s, lane);
                h = dfw_add(h, dfw_norm(df{__ldcg(&v.parth[idx * 4]), __ldcg(&v.partl[idx * 4])}, __ldcg(&v.parte[idx])));
            }
            chain_put(cs->tmph, cs->tmpl, cs->tmpe, lane, h);
            chain_put(cs->hh[slot], cs->hl[slot], cs->he[slot], lane, dfw_zero());
            __syncwarp();
            const dfw gh = dot_row_vec(&T[1], lane, cs->tmph, cs->tmpl, cs->tmpe, 0, lane + 1);
            chain_put(cs->ghh, cs->ghl, cs->ghe, lane, gh);
        }
        __syncthreads();
        if (cs->abort) return;
        if (tid < 32) {
            cs->pvh[tid] = cs->xh[tid];
            cs->pvl[tid] = cs->xl[tid];
            cs->pve[tid] = cs->xe[tid];
        }
        __syncthreads();
    }
}

// Backward chain block.  Shared tiles: T[0] = P_J, T[1] = G_{J-1}, T[2..W-1] = M_{J,J-m}.
__device__ void xchain_backward(const XView& v, DfwTile* T, ChainS* cs)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int* flag_chain = v.flags + v.nb;
    const int* flag_part = v.flags + 2 * v.nb + v.nb * v.S;
    const int W = v.W;
    if (tid == 0) cs->abort = 0;
    for (int m = 0; m < W; ++m)
        if (tid < 32) chain_put(cs->hh[m], cs->hl[m], cs->he[m], tid, dfw_zero());
    const int nbl = v.nb - 1;
    for (int J = nbl; J >= 0; --J) {
        if (J < nbl) stage_block(&T[0], v.Ph + (size_t)J * 1024, v.Pl + (size_t)J * 1024, v.Pe + (size_t)J * 1024);
        else stage_block(&T[0], v.Gh + (size_t)J * 1024, v.Gl + (size_t)J * 1024, v.Ge + (size_t)J * 1024);
        if (J >= 1)
            stage_block(&T[1], v.Gh + (size_t)(J - 1) * 1024, v.Gl + (size_t)(J - 1) * 1024, v.Ge + (size_t)(J - 1) * 1024);
        for (int m = 2; m < W; ++m)
            if (J - m >= 0) {
                const long long t = xdf_tile_index(v, J, J - m);
                stage_block(&T[m], v.Mh + t * 1024, v.Ml + t * 1024, v.Me + t * 1024);
            }
        __syncthreads();
        if (J == nbl) {
            // c_last = G^T e_{Nloc}: row Nloc of G
            if (w == 0) chain_put(cs->xh, cs->xl, cs->xe, lane, tile_get(&T[0], v.N - 32 * nbl, lane));
        } else {
            const dfw p = dot_col_vec(&T[0], lane, cs->pvh, cs->pvl, cs->pve, 4 * w, 4 * w + 4);
            chain_put(cs->rh[w], cs->rl[w], cs->re[w], lane, p);
            __syncthreads();
            if (w == 0) {
                dfw s = chain_get(cs->ghh, cs->ghl, cs->ghe, lane);
                for (int q = 0; q < XDF_WARPS; ++q) s = dfw_add(s, chain_get(cs->rh[q], cs->rl[q], cs->re[q], lane));
                chain_put(cs->xh, cs->xl, cs->xe, lane, s);
            }
        }
        if (w == 0) {
            const int n = 32 * J + lane;
            v.ch[n] = cs->xh[lane];
            v.cl[n] = cs->xl[lane];
            v.ce[n] = cs->xe[lane];
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release(&flag_chain[J], 1);
        }
        __syncthreads();
        // band: hb_{J-m} += M_{J,J-m}^T c_J
        if (w + 2 < W && J - (w + 2) >= 0) {
            const int m = w + 2;
            const dfw p = dot_col_vec(&T[m], lane, cs->xh, cs->xl, cs->xe, 0, 32);
            const int slot = (J - m) % W;
            chain_put(cs->hh[slot], cs->hl[slot], cs->he[slot], lane,
                      dfw_add(chain_get(cs->hh[slot], cs->hl[slot], cs->he[slot], lane), p));
        }
        if (w == XDF_WARPS - 1 && J >= 1) {
            const int Jn = J - 1, slot = Jn % W;
            dfw h = chain_get(cs->hh[slot], cs->hl[slot], cs->he[slot], lane);
            const int ns = min(v.S, v.nb - Jn - W);
            for (int s = 0; s < ns; ++s) {
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_part[Jn * v.S + s], 1, v.err, v.spin_limit, 0x520000 + Jn);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                const size_t idx = xpart_index(v, 1, Jn, s, lane);
                h = dfw_add(h, dfw_norm(df{__ldcg(&v.parth[idx * 4]), __ldcg(&v.partl[idx * 4])}, __ldcg(&v.parte[idx])));
            }
            chain_put(cs->tmph, cs->tmpl, cs->tmpe, lane, h);
            chain_put(cs->hh[slot], cs->hl[slot], cs->he[slot], lane, dfw_zero());
            __syncwarp();
            // (G^T h)[r] = sum_{t >= r} G[t][r] h[t]
            const dfw gh = dot_col_vec(&T[1], lane, cs->tmph, cs->tmpl, cs->tmpe, lane, 32);
            chain_put(cs->ghh, cs->ghl, cs->ghe, lane, gh);
        }
        __syncthreads();
        if (cs->abort) return;
        if (tid < 32) {
            cs->pvh[tid] = cs->xh[tid];
            cs->pvl[tid] = cs->xl[tid];
            cs->pve[tid] = cs->xe[tid];
        }
        __syncthreads();
    }
}

// Forward helper: items (J, s): row block J, column blocks I = s, s+S, ... <= J - W.
__device__ void xhelper_forward(const XView& v, DfwTile* T, WeightSmem* Ws, ChainS* cs, const float2* tab, int h)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int* flag_chain = v.flags;
    int* flag_part = v.flags + 2 * v.nb;
    DfwTile* s = &T[w];
    WeightSmem* ws = &Ws[w];
    if (tid == 0) cs->abort = 0;
    __syncthreads();
    long long q = 0;
    for (int J = v.W; J < v.nb; ++J) {
        const int ns = min(v.S, J - v.W + 1);
        for (int si = 0; si < ns; ++si, ++q) {
            if (q % v.n_help_f != h) continue;
            const int count = (J - v.W - si) / v.S + 1;
            DVAcc acc = dv_zero();
            for (int mm = w; mm < count; mm += XDF_WARPS) {
                const int I = si + mm * v.S;
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_chain[I], 1, v.err, v.spin_limit, 0x530000 + I);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                load_wf(v, ws, I, lane);
                get_tile_warp(v, s, J, I, lane, tab);
                __syncwarp();
                const DVAcc p = weighted_rows(s, ws, lane, v.d);
                dv_add(acc, p);
                __syncwarp();
            }
            cs->hm[w][lane] = acc;
            __syncthreads();
            if (cs->abort) return;
            if (w == 0) {
                DVAcc t = dv_zero();
                for (int q2 = 0; q2 < XDF_WARPS; ++q2) dv_add(t, cs->hm[q2][lane]);
                store_dv(v.parth, v.partl, v.parte, xpart_index(v, 0, J, si, lane), t);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&flag_part[J * v.S + si], 1);
            }
            __syncthreads();
        }
    }
}

// Backward helper: items (I, s): column block I, row blocks J = I+W+s, I+W+s+S, ... < nb.
__device__ void xhelper_backward(const XView& v, DfwTile* T, WeightSmem* Ws, ChainS* cs, const float2* tab, int h)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int* flag_chain = v.flags + v.nb;
    int* flag_part = v.flags + 2 * v.nb + v.nb * v.S;
    DfwTile* s = &T[w];
    WeightSmem* ws = &Ws[w];
    if (tid == 0) cs->abort = 0;
    __syncthreads();
    long long q = 0;
    for (int I = v.nb - 1 - v.W; I >= 0; --I) {
        const int ns = min(v.S, v.nb - I - v.W);
        for (int si = 0; si < ns; ++si, ++q) {
            if (q % v.n_help_b != h) continue;
            const int first = I + v.W + si;
            const int count = (v.nb - 1 - first) / v.S + 1;
            DVAcc acc = dv_zero();
            for (int mm = w; mm < count; mm += XDF_WARPS) {
                const int J = first + mm * v.S;
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_chain[J], 1, v.err, v.spin_limit, 0x540000 + J);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                load_wb(v, ws, J, lane);
                get_tile_warp(v, s, J, I, lane, tab);
                __syncwarp();
                const DVAcc p = weighted_cols(s, ws, lane, v.d);
                dv_add(acc, p);
                __syncwarp();
            }
            cs->hm[w][lane] = acc;
            __syncthreads();
            if (cs->abort) return;
            if (w == 0) {
                DVAcc t = dv_zero();
                for (int q2 = 0; q2 < XDF_WARPS; ++q2) dv_add(t, cs->hm[q2][lane]);
                store_dv(v.parth, v.partl, v.parte, xpart_index(v, 1, I, si, lane), t);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&flag_part[I * v.S + si], 1);
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(XDF_THREADS, 1) xdf_recursion_kernel(XView v)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfwTile* T = reinterpret_cast<DfwTile*>(smem_raw);
    WeightSmem* Ws = reinterpret_cast<WeightSmem*>(smem_raw + XDF_WARPS * sizeof(DfwTile));
    ChainS* cs = reinterpret_cast<ChainS*>(smem_raw + XDF_WARPS * sizeof(DfwTile) + XDF_WARPS * sizeof(WeightSmem));
    // the float2 table needs 8-byte alignment: round its offset up to 16 bytes
    const size_t tab_off = (XDF_WARPS * sizeof(DfwTile) + XDF_WARPS * sizeof(WeightSmem) + sizeof(ChainS) + 15) & ~(size_t)15;
    float2* tab = reinterpret_cast<float2*>(smem_raw + tab_off);
    load_tab_smem(tab, v.tab);
    __syncthreads();
    const int bid = blockIdx.x;
    if (bid == 0) xchain_forward(v, T, cs);
    else if (bid == 1) xchain_backward(v, T, cs);
    else if (bid - 2 < v.n_help_f) xhelper_forward(v, T, Ws, cs, tab, bid - 2);
    else xhelper_backward(v, T, Ws, cs, tab, bid - 2 - v.n_help_f);
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
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int blk = blockIdx.x, dir = blockIdx.y;
    DVAcc a = dv_zero();
    if (dir == 0) {
        const int J = blk, I = blk - w;
        if (I >= 0) {
            load_wf(v, &Ws[w], I, lane);
            get_tile_warp(v, &T[w], J, I, lane, tab);
            __syncwarp();
            a = weighted_rows(&T[w], &Ws[w], lane, v.d);
        }
    } else {
        const int I = blk, J = blk + w;
        if (J < v.nb) {
            load_wb(v, &Ws[w], J, lane);
            get_tile_warp(v, &T[w], J, I, lane, tab);
            __syncwarp();
            a = weighted_cols(&T[w], &Ws[w], lane, v.d);
        }
    }
    hm[w * 32 + lane] = a;
    __syncthreads();
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
    const size_t tab_off = (XDF_WARPS * sizeof(DfwTile) + XDF_WARPS * sizeof(WeightSmem) + sizeof(ChainS) + 15) & ~(size_t)15;
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
