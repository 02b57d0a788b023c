// Exchange kernels for sm_103a: factor table, persistent recursion, band
// sums and endpoint-force assembly (arXiv 2404.02628, Sec. III).  The
// factorised equations are stated in pimd_exchange.cuh.
#include <math.h>

#include "pimd_exchange.cuh"

namespace {

__device__ __forceinline__ double ex_a(const ExchView& v, int c, int i) { return v.a[(size_t)c * v.lda + i]; }
__device__ __forceinline__ double ex_b(const ExchView& v, int c, int k) { return v.b[(size_t)c * v.ldb + k]; }

// g(i,k) = kappa |r_i^P - r_k^1|^2
__device__ __forceinline__ double ex_g(const ExchView& v, int i, int k)
{
    double s = 0.0;
    for (int c = 0; c < v.d; ++c) {
        double x = ex_a(v, c, i) - ex_b(v, c, k);
        s = fma(x, x, s);
    }
    return v.kappa * s;
}

struct ExSlot {  // one staged 32x32 tile with its 32 weights
    double Km[32 * EX_LD];
    double wm[32];
    double wv[3][32];
    int Ke[32 * EX_LD];
    int we[32];
};

struct ChainSmem {
    double red_m[EX_WARPS][32];
    int red_e[EX_WARPS][32];
    double col_m[32];  // forward: y of the previous column block; backward: z of the previous row block
    int col_e[32];
    double hm[EX_WARPS][32][4];  // helper cross-warp merge
    int he[EX_WARPS][32];
    int abort;
};

struct VAcc {
    double s;
    double v[3];
    int e;
};

__device__ __forceinline__ VAcc vacc_zero()
{
    VAcc a;
    a.s = 0.0;
    a.v[0] = a.v[1] = a.v[2] = 0.0;
    a.e = WEF_ZERO_E;
    return a;
}

// A += (S, V) * 2^E; S >= 0 is the scalar row/column sum, V the weighted sums.
__device__ __forceinline__ void vacc_add(VAcc& A, double S, const double* V, int E)
{
    if (!(S > 0.0)) {
        if (S != 0.0) A.s = S;  // NaN propagates
        return;
    }
    if (A.s == 0.0) {
        A.s = S;
        A.v[0] = V[0]; A.v[1] = V[1]; A.v[2] = V[2];
        A.e = E;
    } else if (A.e >= E) {
        double f = pow2i(E - A.e);
        A.s = fma(S, f, A.s);
#pragma unroll
        for (int c = 0; c < 3; ++c) A.v[c] = fma(V[c], f, A.v[c]);
    } else {
        double f = pow2i(A.e - E);
        A.s = fma(A.s, f, S);
#pragma unroll
        for (int c = 0; c < 3; ++c) A.v[c] = fma(A.v[c], f, V[c]);
        A.e = E;
    }
    int ex = ((__double2hiint(A.s) >> 20) & 0x7FF) - 1023;
    if (ex != 0 && A.s > 0.0) {
        double f = pow2i(-ex);
        A.s *= f;
#pragma unroll
        for (int c = 0; c < 3; ++c) A.v[c] *= f;
        A.e += ex;
    }
}

// Stage tile (J,I) into slot s with all threads of the block.
__device__ __forceinline__ void stage_tile_block(const ExchView& v, ExSlot* s, int J, int I)
{
    const long long t = ex_tile_index(v, J, I);
    const double* Km = v.Km + t * 1024;
    const int* Ke = v.Ke + t * 1024;
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
        int k = e >> 5, i = e & 31;
        s->Km[k * EX_LD + i] = Km[e];
        s->Ke[k * EX_LD + i] = Ke[e];
    }
}

// Stage or compute tile (J,I) into slot s with one warp.
__device__ __forceinline__ void stage_tile_warp(const ExchView& v, ExSlot* s, int J, int I, int lane)
{
    if (v.store || J - I <= 1) {
        const long long t = ex_tile_index(v, J, I);
        const double* Km = v.Km + t * 1024;
        const int* Ke = v.Ke + t * 1024;
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            s->Km[k * EX_LD + lane] = Km[k * 32 + lane];
            s->Ke[k * EX_LD + lane] = Ke[k * 32 + lane];
        }
        return;
    }
    // recompute: lane = row i of block J; columns broadcast by shuffles
    const int i = 32 * J + lane, kk = 32 * I + lane;
    double ai[3] = {0.0, 0.0, 0.0}, bk[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < v.d; ++c) {
        if (i < v.N) ai[c] = ex_a(v, c, i);
        if (kk < v.N) bk[c] = ex_b(v, c, kk);
    }
    for (int k = 0; k < 32; ++k) {
        double q = 0.0;
        for (int c = 0; c < v.d; ++c) {
            double x = ai[c] - __shfl_sync(0xffffffffu, bk[c], k);
            q = fma(x, x, q);
        }
        Wef w = (i < v.N && 32 * I + k <= i) ? wef_exp(-v.kappa * q) : wef_zero();
        s->Km[k * EX_LD + lane] = w.m;
        s->Ke[k * EX_LD + lane] = w.e;
    }
}

// Row sums of a staged tile for row `lane`: S = sum_k K y_k, V = sum_k K y_k b_k,
// both relative to 2^E.
__device__ __forceinline__ void tile_rows(const ExSlot* s, int lane, double& S, double* V, int& E)
{
    int Em = WEF_ZERO_E;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) Em = max(Em, s->Ke[k * EX_LD + lane] + s->we[k]);
    S = 0.0;
    V[0] = V[1] = V[2] = 0.0;
    E = Em;
    if (Em <= WEF_ZERO_E / 2) return;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
        double ks = scale_down(s->Km[k * EX_LD + lane], s->Ke[k * EX_LD + lane] + s->we[k] - Em);
        S = fma(ks, s->wm[k], S);
        V[0] = fma(ks, s->wv[0][k], V[0]);
        V[1] = fma(ks, s->wv[1][k], V[1]);
        V[2] = fma(ks, s->wv[2][k], V[2]);
    }
}

// Column sums of a staged tile for column `lane`: S = sum_i K z_i, V = sum_i K z_i a_i.
__device__ __forceinline__ void tile_cols(const ExSlot* s, int lane, double& S, double* V, int& E)
{
    int Em = WEF_ZERO_E;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) Em = max(Em, s->Ke[lane * EX_LD + i] + s->we[i]);
    S = 0.0;
    V[0] = V[1] = V[2] = 0.0;
    E = Em;
    if (Em <= WEF_ZERO_E / 2) return;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        double ks = scale_down(s->Km[lane * EX_LD + i], s->Ke[lane * EX_LD + i] + s->we[i] - Em);
        S = fma(ks, s->wm[i], S);
        V[0] = fma(ks, s->wv[0][i], V[0]);
        V[1] = fma(ks, s->wv[1][i], V[1]);
        V[2] = fma(ks, s->wv[2][i], V[2]);
    }
}

// Weights of a column block I for row sums: y[k] and y[k] b_k (zero past N).
__device__ __forceinline__ void load_weights_fwd(const ExchView& v, ExSlot* s, int I, int lane)
{
    const int k = 32 * I + lane;
    double m = 0.0;
    int e = WEF_ZERO_E;
    if (k < v.N) {
        m = __ldcg(&v.y_m[k]);
        e = __ldcg(&v.y_e[k]);
    }
    s->wm[lane] = m;
    s->we[lane] = e;
    for (int c = 0; c < 3; ++c) s->wv[c][lane] = (c < v.d && k < v.N) ? m * ex_b(v, c, k) : 0.0;
}

// Weights of a row block J for column sums: z[i] and z[i] a_i (zero past N).
__device__ __forceinline__ void load_weights_bwd(const ExchView& v, ExSlot* s, int J, int lane)
{
    const int i = 32 * J + lane;
    double m = 0.0;
    int e = WEF_ZERO_E;
    if (i < v.N) {
        m = __ldcg(&v.z_m[i]);
        e = __ldcg(&v.z_e[i]);
    }
    s->wm[lane] = m;
    s->we[lane] = e;
    for (int c = 0; c < 3; ++c) s->wv[c][lane] = (c < v.d && i < v.N) ? m * ex_a(v, c, i) : 0.0;
}

__device__ __forceinline__ size_t part_index(const ExchView& v, int dir, int blk, int s, int lane)
{
    return ((((size_t)dir * v.nb + blk) * v.S + s) << 5) + lane;
}

__device__ __forceinline__ size_t band_index(const ExchView& v, int dir, int blk, int which, int lane)
{
    return ((((size_t)dir * v.nb + blk) * 2 + which) << 5) + lane;
}

__device__ __forceinline__ void store_vacc(double* m, int* e, size_t idx, const VAcc& a)
{
    m[idx * 4 + 0] = a.s;
    m[idx * 4 + 1] = a.v[0];
    m[idx * 4 + 2] = a.v[1];
    m[idx * 4 + 3] = a.v[2];
    e[idx] = a.e;
}

__device__ __forceinline__ void add_stored_vacc(VAcc& acc, const double* m, const int* e, size_t idx)
{
    double V[3] = {__ldcg(&m[idx * 4 + 1]), __ldcg(&m[idx * 4 + 2]), __ldcg(&m[idx * 4 + 3])};
    vacc_add(acc, __ldcg(&m[idx * 4]), V, __ldcg(&e[idx]));
}

// ------------------------------------------------------------------------
// Forward chain: y[i+1] = rho[i] * sum_{k<=i} K[i][k] y[k], one 32-row block
// at a time.  Helper partials (column blocks <= J-2) and the subdiagonal tile
// are summed first; the diagonal tile is then walked serially by one warp.

__device__ void chain_forward(const ExchView& v, ExSlot* slots, ChainSmem* cs)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int* flag_chain = v.flags;
    const int* flag_part = v.flags + 2 * v.nb;
    ExSlot* sd = &slots[0];
    ExSlot* ss = &slots[1];
    Wef ycarry = Wef{1.0, 0};  // y[0]
    if (tid == 0) cs->abort = 0;
    for (int J = 0; J < v.nb; ++J) {
        stage_tile_block(v, sd, J, J);
        if (J > 0) stage_tile_block(v, ss, J, J - 1);
        block_sync();
        if (J > 0) {
            int Em = WEF_ZERO_E;
            for (int q = 0; q < 4; ++q) {
                int k = 4 * w + q;
                Em = max(Em, ss->Ke[k * EX_LD + lane] + cs->col_e[k]);
            }
            double s = 0.0;
            if (Em > WEF_ZERO_E / 2)
                for (int q = 0; q < 4; ++q) {
                    int k = 4 * w + q;
                    s = fma(scale_down(ss->Km[k * EX_LD + lane], ss->Ke[k * EX_LD + lane] + cs->col_e[k] - Em),
                            cs->col_m[k], s);
                }
            cs->red_m[w][lane] = s;
            cs->red_e[w][lane] = Em;
        }
        block_sync();
        if (w == 0) {
            Wef acc = wef_zero();
            const int ns = min(v.S, J - 1);
            for (int s = 0; s < ns; ++s) {
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_part[J * v.S + s], 1, v.err, v.spin_limit, 0x100000 + J);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                size_t idx = part_index(v, 0, J, s, lane);
                acc = wef_add(acc, wef_norm(__ldcg(&v.part_m[idx * 4]), __ldcg(&v.part_e[idx])));
            }
            if (!cs->abort) {
                if (J > 0)
                    for (int q = 0; q < EX_WARPS; ++q) acc = wef_add(acc, wef_norm(cs->red_m[q][lane], cs->red_e[q][lane]));
                const int i = 32 * J + lane;
                const Wef rho = (i < v.N) ? Wef{v.rho_m[i], v.rho_e[i]} : wef_zero();
                const int nrows = min(32, v.N - 32 * J);
                Wef yk = ycarry;
                for (int tp = 0; tp < nrows; ++tp) {
                    if (lane == tp) {
                        cs->col_m[tp] = yk.m;
                        cs->col_e[tp] = yk.e;
                        v.y_m[32 * J + tp] = yk.m;
                        v.y_e[32 * J + tp] = yk.e;
                    }
                    if (lane >= tp) acc = wef_add(acc, wef_mul(Wef{sd->Km[tp * EX_LD + lane], sd->Ke[tp * EX_LD + lane]}, yk));
                    Wef yn = wef_mul(rho, acc);
                    yk.m = __shfl_sync(0xffffffffu, yn.m, tp);
                    yk.e = __shfl_sync(0xffffffffu, yn.e, tp);
                }
                if (lane >= nrows) {
                    cs->col_m[lane] = 0.0;
                    cs->col_e[lane] = WEF_ZERO_E;
                }
                ycarry = yk;
                if (32 * J + nrows == v.N && lane == 0) {
                    v.y_m[v.N] = yk.m;
                    v.y_e[v.N] = yk.e;
                }
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&flag_chain[J], 1);
            }
        }
        block_sync();
        if (cs->abort) return;
    }
}

// Backward chain: c[k] = sum_{i>=k} K[i][k] z[i], z[i] = rho[i] c[i+1], one
// 32-column block at a time from the top.
__device__ void chain_backward(const ExchView& v, ExSlot* slots, ChainSmem* cs)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int* flag_chain = v.flags + v.nb;
    const int* flag_part = v.flags + 2 * v.nb + v.nb * v.S;
    ExSlot* sd = &slots[0];
    ExSlot* ss = &slots[1];
    Wef zcarry = wef_zero();
    if (tid == 0) {
        cs->abort = 0;
        v.c_m[v.N] = 1.0;
        v.c_e[v.N] = 0;
    }
    for (int I = v.nb - 1; I >= 0; --I) {
        stage_tile_block(v, sd, I, I);
        if (I + 1 < v.nb) stage_tile_block(v, ss, I + 1, I);
        block_sync();
        if (I + 1 < v.nb) {
            int Em = WEF_ZERO_E;
            for (int q = 0; q < 4; ++q) {
                int i = 4 * w + q;
                Em = max(Em, ss->Ke[lane * EX_LD + i] + cs->col_e[i]);
            }
            double s = 0.0;
            if (Em > WEF_ZERO_E / 2)
                for (int q = 0; q < 4; ++q) {
                    int i = 4 * w + q;
                    s = fma(scale_down(ss->Km[lane * EX_LD + i], ss->Ke[lane * EX_LD + i] + cs->col_e[i] - Em),
                            cs->col_m[i], s);
                }
            cs->red_m[w][lane] = s;
            cs->red_e[w][lane] = Em;
        }
        block_sync();
        if (w == 0) {
            Wef acc = wef_zero();
            const int ns = min(v.S, v.nb - 2 - I);
            for (int s = 0; s < ns; ++s) {
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_part[I * v.S + s], 1, v.err, v.spin_limit, 0x200000 + I);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                size_t idx = part_index(v, 1, I, s, lane);
                acc = wef_add(acc, wef_norm(__ldcg(&v.part_m[idx * 4]), __ldcg(&v.part_e[idx])));
            }
            if (!cs->abort) {
                if (I + 1 < v.nb)
                    for (int q = 0; q < EX_WARPS; ++q) acc = wef_add(acc, wef_norm(cs->red_m[q][lane], cs->red_e[q][lane]));
                const int k = 32 * I + lane;
                const Wef rho_prev = (k >= 1 && k - 1 < v.N) ? Wef{v.rho_m[k - 1], v.rho_e[k - 1]} : wef_zero();
                const int top = min(32 * I + 31, v.N - 1);
                Wef zk = (top == v.N - 1) ? Wef{v.rho_m[v.N - 1], v.rho_e[v.N - 1]} : zcarry;
                for (int i = top; i >= 32 * I; --i) {
                    const int tp = i - 32 * I;
                    if (lane == tp) {
                        cs->col_m[tp] = zk.m;
                        cs->col_e[tp] = zk.e;
                        v.z_m[i] = zk.m;
                        v.z_e[i] = zk.e;
                    }
                    if (lane <= tp) acc = wef_add(acc, wef_mul(Wef{sd->Km[lane * EX_LD + tp], sd->Ke[lane * EX_LD + tp]}, zk));
                    if (lane == tp) {
                        v.c_m[i] = acc.m;
                        v.c_e[i] = acc.e;
                    }
                    Wef zn = wef_mul(rho_prev, acc);
                    zk.m = __shfl_sync(0xffffffffu, zn.m, tp);
                    zk.e = __shfl_sync(0xffffffffu, zn.e, tp);
                }
                if (lane > top - 32 * I) {
                    cs->col_m[lane] = 0.0;
                    cs->col_e[lane] = WEF_ZERO_E;
                }
                zcarry = zk;
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&flag_chain[I], 1);
            }
        }
        block_sync();
        if (cs->abort) return;
    }
}

// Forward helper: items (J, s) = row block J, column blocks I = s, s+S, ... <= J-2.
__device__ void helper_forward(const ExchView& v, ExSlot* slots, ChainSmem* cs, int h)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int* flag_chain = v.flags;
    int* flag_part = v.flags + 2 * v.nb;
    ExSlot* s = &slots[w];
    if (tid == 0) cs->abort = 0;
    block_sync();
    long long q = 0;
    for (int J = 2; J < v.nb; ++J) {
        const int ns = min(v.S, J - 1);
        for (int si = 0; si < ns; ++si, ++q) {
            if (q % v.n_help_f != h) continue;
            const int count = (J - 2 - si) / v.S + 1;
            VAcc acc = vacc_zero();
            for (int mm = w; mm < count; mm += EX_WARPS) {
                const int I = si + mm * v.S;
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_chain[I], 1, v.err, v.spin_limit, 0x300000 + I);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                load_weights_fwd(v, s, I, lane);
                stage_tile_warp(v, s, J, I, lane);
                __syncwarp();
                double S, V[3];
                int E;
                tile_rows(s, lane, S, V, E);
                vacc_add(acc, S, V, E);
                __syncwarp();
            }
            cs->hm[w][lane][0] = acc.s;
            cs->hm[w][lane][1] = acc.v[0];
            cs->hm[w][lane][2] = acc.v[1];
            cs->hm[w][lane][3] = acc.v[2];
            cs->he[w][lane] = acc.e;
            block_sync();
            if (cs->abort) return;
            if (w == 0) {
                VAcc t = vacc_zero();
                for (int q2 = 0; q2 < EX_WARPS; ++q2) vacc_add(t, cs->hm[q2][lane][0], &cs->hm[q2][lane][1], cs->he[q2][lane]);
                store_vacc(v.part_m, v.part_e, part_index(v, 0, J, si, lane), t);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&flag_part[J * v.S + si], 1);
            }
            block_sync();
        }
    }
}

// Backward helper: items (I, s) = column block I, row blocks J = I+2+s, I+2+s+S, ... < nb.
__device__ void helper_backward(const ExchView& v, ExSlot* slots, ChainSmem* cs, int h)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int* flag_chain = v.flags + v.nb;
    int* flag_part = v.flags + 2 * v.nb + v.nb * v.S;
    ExSlot* s = &slots[w];
    if (tid == 0) cs->abort = 0;
    block_sync();
    long long q = 0;
    for (int I = v.nb - 3; I >= 0; --I) {
        const int ns = min(v.S, v.nb - 2 - I);
        for (int si = 0; si < ns; ++si, ++q) {
            if (q % v.n_help_b != h) continue;
            const int first = I + 2 + si;
            const int count = (v.nb - 1 - first) / v.S + 1;
            VAcc acc = vacc_zero();
            for (int mm = w; mm < count; mm += EX_WARPS) {
                const int J = first + mm * v.S;
                int ok = 1;
                if (lane == 0) ok = wait_flag(&flag_chain[J], 1, v.err, v.spin_limit, 0x400000 + J);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) cs->abort = 1;
                    break;
                }
                load_weights_bwd(v, s, J, lane);
                stage_tile_warp(v, s, J, I, lane);
                __syncwarp();
                double S, V[3];
                int E;
                tile_cols(s, lane, S, V, E);
                vacc_add(acc, S, V, E);
                __syncwarp();
            }
            cs->hm[w][lane][0] = acc.s;
            cs->hm[w][lane][1] = acc.v[0];
            cs->hm[w][lane][2] = acc.v[1];
            cs->hm[w][lane][3] = acc.v[2];
            cs->he[w][lane] = acc.e;
            block_sync();
            if (cs->abort) return;
            if (w == 0) {
                VAcc t = vacc_zero();
                for (int q2 = 0; q2 < EX_WARPS; ++q2) vacc_add(t, cs->hm[q2][lane][0], &cs->hm[q2][lane][1], cs->he[q2][lane]);
                store_vacc(v.part_m, v.part_e, part_index(v, 1, I, si, lane), t);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&flag_part[I * v.S + si], 1);
            }
            block_sync();
        }
    }
}

// ------------------------------------------------------------------------
// Kernels

__global__ void __launch_bounds__(256) exch_prep_kernel(ExchView v)
{
    __shared__ double red[32 * 2];
    double acc[2] = {0.0, 0.0};
    const int nbp = v.nb * 32;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbp; i += gridDim.x * blockDim.x) {
        Wef r = wef_zero();
        if (i < v.N) {
            double gl = (i < v.N - 1) ? ex_g(v, i, i + 1) : 0.0;
            double lr = gl - log((double)(i + 1));  // ln of exp(g(i,i+1))/(i+1)
            if (!v.xi_zero) r = wef_exp(lr - v.log_xi);
            acc[0] += gl;
            if (v.xi_zero) acc[1] += lr - ex_g(v, i, i);
        }
        v.rho_m[i] = r.m;
        v.rho_e[i] = r.e;
    }
    const int nflags = 2 * v.nb + 2 * v.nb * v.S;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nflags; j += gridDim.x * blockDim.x) v.flags[j] = 0;
    block_reduce<2>(acc, red);
    if (threadIdx.x == 0) {
        v.lsum[blockIdx.x * 2 + 0] = acc[0];
        v.lsum[blockIdx.x * 2 + 1] = acc[1];
    }
}

__global__ void __launch_bounds__(256) exch_table_kernel(ExchView v, long long ntiles)
{
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int J, I;
        if (v.store) {
            J = (int)floor((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
            while ((long long)J * (J + 1) / 2 > t) --J;
            while ((long long)(J + 1) * (J + 2) / 2 <= t) ++J;
            I = (int)(t - (long long)J * (J + 1) / 2);
        } else if (t < v.nb) {
            J = I = (int)t;
        } else {
            J = (int)(t - v.nb) + 1;
            I = J - 1;
        }
        double* Km = v.Km + t * 1024;
        int* Ke = v.Ke + t * 1024;
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int i = 32 * J + (e & 31), k = 32 * I + (e >> 5);
            Wef w = wef_zero();
            if (i < v.N && k <= i) w = wef_exp(-ex_g(v, i, k));
            Km[e] = w.m;
            Ke[e] = w.e;
        }
    }
}

__global__ void __launch_bounds__(EX_THREADS, 1) exch_recursion_kernel(ExchView v)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ExSlot* slots = reinterpret_cast<ExSlot*>(smem_raw);
    ChainSmem* cs = reinterpret_cast<ChainSmem*>(smem_raw + EX_WARPS * sizeof(ExSlot));
    const int bid = blockIdx.x;
    if (bid == 0) chain_forward(v, slots, cs);
    else if (bid == 1) chain_backward(v, slots, cs);
    else if (bid - 2 < v.n_help_f) helper_forward(v, slots, cs, bid - 2);
    else helper_backward(v, slots, cs, bid - 2 - v.n_help_f);
}

// Band sums (diagonal and subdiagonal tiles) of the row/column weighted sums,
// once the chains are done.  Block (blk, dir), warp 0 = diagonal tile, warp 1 = subdiagonal.
__global__ void __launch_bounds__(64) exch_band_kernel(ExchView v)
{
    __shared__ ExSlot slots[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int blk = blockIdx.x, dir = blockIdx.y;
    ExSlot* s = &slots[w];
    VAcc a = vacc_zero();
    double S = 0.0, V[3] = {0.0, 0.0, 0.0};
    int E = WEF_ZERO_E;
    if (dir == 0) {
        const int J = blk, I = blk - w;
        if (I >= 0) {
            load_weights_fwd(v, s, I, lane);
            stage_tile_warp(v, s, J, I, lane);
            __syncwarp();
            tile_rows(s, lane, S, V, E);
        }
    } else {
        const int I = blk, J = blk + w;
        if (J < v.nb) {
            load_weights_bwd(v, s, J, lane);
            stage_tile_warp(v, s, J, I, lane);
            __syncwarp();
            tile_cols(s, lane, S, V, E);
        }
    }
    vacc_add(a, S, V, E);
    store_vacc(v.band_m, v.band_e, band_index(v, dir, blk, w, lane), a);
}

// Endpoint forces (Sec. III exterior-bead formulas in the factorised form).
__global__ void __launch_bounds__(256) exch_finalize_kernel(ExchView v, FinalizeOut o)
{
    __shared__ double red[32];
    double esum[1] = {0.0};
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < v.N) {
        double a[3] = {0.0, 0.0, 0.0}, b[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < v.d; ++c) {
            a[c] = ex_a(v, c, l);
            b[c] = ex_b(v, c, l);
        }
        double rowtot, coltot, PB[3], PA[3], link, linkin;
        if (v.xi_zero) {
            rowtot = coltot = 1.0;
            for (int c = 0; c < 3; ++c) {
                PB[c] = b[c];
                PA[c] = a[c];
            }
            link = linkin = 0.0;
        } else {
            const int blk = l >> 5, lane = l & 31;
            VAcc R = vacc_zero(), C = vacc_zero();
            for (int s = 0; s < min(v.S, blk - 1); ++s) add_stored_vacc(R, v.part_m, v.part_e, part_index(v, 0, blk, s, lane));
            add_stored_vacc(R, v.band_m, v.band_e, band_index(v, 0, blk, 0, lane));
            if (blk > 0) add_stored_vacc(R, v.band_m, v.band_e, band_index(v, 0, blk, 1, lane));
            for (int s = 0; s < min(v.S, v.nb - 2 - blk); ++s) add_stored_vacc(C, v.part_m, v.part_e, part_index(v, 1, blk, s, lane));
            add_stored_vacc(C, v.band_m, v.band_e, band_index(v, 1, blk, 0, lane));
            if (blk + 1 < v.nb) add_stored_vacc(C, v.band_m, v.band_e, band_index(v, 1, blk, 1, lane));
            const Wef Z = Wef{v.y_m[v.N], v.y_e[v.N]};
            const Wef iZ = wef_norm(1.0 / Z.m, -Z.e);
            const Wef yl = Wef{v.y_m[l], v.y_e[l]}, yl1 = Wef{v.y_m[l + 1], v.y_e[l + 1]};
            const Wef cl = Wef{v.c_m[l], v.c_e[l]}, cl1 = Wef{v.c_m[l + 1], v.c_e[l + 1]};
            const Wef zl = Wef{v.z_m[l], v.z_e[l]};
            rowtot = wef_to_double(wef_mul(wef_mul(yl1, cl1), iZ));
            coltot = wef_to_double(wef_mul(wef_mul(yl, cl), iZ));
            Wef fr = wef_mul(zl, iZ);
            fr.e += R.e;
            Wef fc = wef_mul(yl, iZ);
            fc.e += C.e;
            const double sr = wef_to_double(fr), sc = wef_to_double(fc);
            for (int c = 0; c < 3; ++c) {
                PB[c] = R.v[c] * sr;
                PA[c] = C.v[c] * sc;
            }
            link = (l < v.N - 1) ? 1.0 - rowtot : 0.0;
            linkin = (l >= 1) ? 1.0 - coltot : 0.0;
        }
        double FP[3], F1[3], e = 0.0;
        for (int c = 0; c < v.d; ++c) {
            const double bn = (l < v.N - 1) ? ex_b(v, c, l + 1) : 0.0;
            const double ap = (l >= 1) ? ex_a(v, c, l - 1) : 0.0;
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
            // a device wait that gave up makes every gradient NaN
            const double gs = *(volatile int*)v.err != 0 ? __longlong_as_double(0x7ff8000000000000LL) : *o.gscale;
            for (int c = 0; c < v.d; ++c) {
                o.g1[(size_t)c * o.ldg + l] = -gs * F1[c];
                o.gP[(size_t)c * o.ldg + l] = -gs * FP[c];
            }
        }
    }
    block_reduce<1>(esum, red);
    if (threadIdx.x == 0 && o.part) o.part[blockIdx.x] = esum[0];
}

// V_ends = sum_{i<N-1} g(i,i+1)/beta - (N ln xi + ln Z)/beta (xi > 0), or with
// the xi = 0 product of the diagonal chain.
// A device wait that gave up during the call (error word set) gives NaN, so
// a caller that cannot synchronise still sees that the value is invalid.
__global__ void exch_vb_value_kernel(ExchView v, int nprep, double* V_out)
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
    double lam = v.xi_zero ? l0 : v.N * v.log_xi + wef_log(Wef{v.y_m[v.N], v.y_e[v.N]});
    *V_out = (gl - lam) / v.beta;
}

}  // namespace

int exch_prep_blocks(int N) { return min(152, (N + 32 + 255) / 256); }
int exch_finalize_blocks(int N) { return (N + 255) / 256; }

size_t exch_recursion_smem() { return EX_WARPS * sizeof(ExSlot) + sizeof(ChainSmem); }

void prof_mark(ProfMarks* pm, const char* name, cudaStream_t st)
{
    if (!pm || pm->n >= 64) return;
    cudaEventRecord(pm->ev[pm->n], st);
    pm->name[pm->n] = name;
    pm->n++;
}

cudaError_t exch_launch_forward(const ExchView& v, cudaStream_t st, int coop, ProfMarks* pm)
{
    exch_prep_kernel<<<exch_prep_blocks(v.N), 256, 0, st>>>(v);
    prof_mark(pm, "exch_prep", st);
    if (v.xi_zero) return cudaGetLastError();
    const long long ntiles = v.store ? (long long)v.nb * (v.nb + 1) / 2 : (long long)(2 * v.nb - 1);
    const int tgrid = (int)min(ntiles, (long long)152 * 64);
    exch_table_kernel<<<tgrid, 256, 0, st>>>(v, ntiles);
    prof_mark(pm, "exch_table", st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = exch_recursion_smem();
    static DeviceOnce attr_once;
    e = device_once(attr_once, [&] {
        return cudaFuncSetAttribute(exch_recursion_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    const int grid = 2 + v.n_help_f + v.n_help_b;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(EX_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = coop ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, exch_recursion_kernel, v);
    prof_mark(pm, "exch_recursion", st);
    return e;
}

cudaError_t exch_launch_adjoint(const ExchView& v, const FinalizeOut& o, int nblk_fin, cudaStream_t st,
                                ProfMarks* pm)
{
    if (!v.xi_zero) {
        exch_band_kernel<<<dim3(v.nb, 2), 64, 0, st>>>(v);
        prof_mark(pm, "exch_band", st);
    }
    exch_finalize_kernel<<<nblk_fin, 256, 0, st>>>(v, o);
    prof_mark(pm, "exch_finalize", st);
    return cudaGetLastError();
}

cudaError_t exch_launch_vb_value(const ExchView& v, int nprep, double* V_out, cudaStream_t st)
{
    exch_vb_value_kernel<<<1, 32, 0, st>>>(v, nprep, V_out);
    return cudaGetLastError();
}
