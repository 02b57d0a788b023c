// Exchange part of the PIMD force field (arXiv 2404.02628, Sec. III) in
// double-float arithmetic with a blocked, look-ahead triangular solve.
//
// With a_i = r_i^P, b_k = r_k^1, g(i,k) = kappa |a_i - b_k|^2 and the row
// constant c_n = g(n-1,n) - ln n - ln xi (c_N = -ln N - ln xi), the matrix
//   M[n][k] = exp(c_n - g(n-1,k)),   1 <= n <= N, 0 <= k < n,
// turns the forward recursion of Sec. III into the unit lower-triangular
// system  y = e_0 + M y  and the backward recursion into its transpose
//   c = e_N + M^T c,  with  W_N = xi^N Z,  Z = y[N] = c[0],
//   V_xi = sum E_int + sum link - (N ln xi + ln Z)/beta,
//   Pr[G(n-1)=k] = M[n][k] y[k] c[n] / Z (k < n),  Pr[G(i)=i+1] = 1 - y[i+1] c[i+1] / Z.
// The endpoint forces need only the weighted sums sum_k M[n][k] y[k] b_k
// (rows) and sum_n M[n][k] c[n] a_{n-1} (columns), accumulated next to the
// solves: the backward recursion is the adjoint of the forward one.
//
// Blocking (32 indices per block, nb blocks):  y_J = G_J sum_{I<J} M_JI y_I with
// G_J = (I - M_JJ)^{-1}; the position-only operators G_J, Q_J = G_J M_{J,J-1}
// and P_J = M_{J+1,J} G_J are built in parallel before the solve, so the
// serial chain does one 32x32 matvec per block:
//   y_J = G_J h_J + Q_J y_{J-1},        h_J = sum_{I<=J-2} M_JI y_I,
//   c_J = G_J^T hb_J + P_J^T c_{J+1},   hb_J = sum_{I>=J+2} M_IJ^T c_I.
// The chain block adds the band tiles I in [J-W+1, J-2] itself (right-looking,
// from values it just produced); helper blocks add I <= J-W and publish
// partial sums through release/acquire flags.  All values are non-negative
// wide-exponent double-floats (dfw), so no sum cancels or overflows.
#pragma once
#include "pimd_df.cuh"
#include "pimd_exchange.cuh"

#define XDF_THREADS 256
#define XDF_WARPS 8
#define XDF_LD 33
#define XDF_MAXW 5

// A 32x32 dfw tile, in global and in shared memory alike: three contiguous
// 4 KB runs (high parts, low parts, exponents), element (r, c) at
// (r << 5) + ((c + r) & 31).  The rotation makes both row walks (lane = r)
// and column walks (lane = c) hit 32 distinct shared-memory banks; the
// contiguity lets one 12 KB bulk copy move a tile.
struct XTile {
    float h[1024];
    float l[1024];
    int e[1024];
};

struct XView {
    int N, nb, npad, d, S, W;
    int store;
    int xi_zero;
    double kappa, ks, beta, log_xi;
    float kap_h, kap_l;          // kappa as a double-float
    const double* a;             // FP64 bead P, component c of particle i at a[c*lda + i]
    const double* b;             // FP64 bead 1
    int lda, ldb;
    float* ah; float* al;        // [3][npad] a_i in double-float
    float* bh; float* bl;        // [3][npad] b_k in double-float
    float* crh; float* crl;      // [npad] row constants c_n
    const float2* tab;           // [256] 2^(j/256) as double-floats
    const double* lnn;           // [npad] ln n (entry 0 unused), filled once per workspace
    XTile* M;                    // factor tiles, index xdf_tile_index
    XTile* G;                    // [nb] (I - M_JJ)^{-1}
    XTile* Q;                    // [nb] G_J M_{J,J-1}
    XTile* P;                    // [nb] M_{J+1,J} G_J
    float* yh; float* yl; int* ye;   // [npad] forward solution y
    float* ch; float* cl; int* ce;   // [npad] backward solution c
    float* uh; float* ul;            // [3][npad] y[k] b_k (mantissa of y times b_k), published with y
    float* wh; float* wl;            // [3][npad] c[n] a_{n-1}, published with c
    float* parth; float* partl; int* parte;  // helper partials [2][nb][S][32] x 4 / x 1
    float* bandh; float* bandl; int* bande;  // band sums [2][nb][32], then diagonal-tile sums [2][nb][32]; x 4 / x 1
    int* flags;                  // [2][nb] chain flags, then [2][nb][S] partial flags
    int* err;
    int spin_limit;
    int n_help_f, n_help_b;
    double* lsum;                // prep partial sums [grid][2]
    double* lam;                 // [2]: ln Z forward and backward (+ N ln xi)
};

__host__ __device__ inline long long xdf_tile_index(const XView& v, int J, int I)
{
    if (v.store) return (long long)J * (J + 1) / 2 + I;
    return (long long)J * v.W + (J - I);
}

__host__ __device__ inline long long xdf_ntiles(int nb, int W, int store)
{
    return store ? (long long)nb * (nb + 1) / 2 : (long long)nb * W;
}

int xdf_prep_blocks(int npad);
int xdf_finalize_blocks(int N);
size_t xdf_recursion_smem(int W);
cudaError_t xdf_upload_table(float2* dev_table, cudaStream_t st);
cudaError_t xdf_fill_lntab(double* dev_lnn, int npad, cudaStream_t st);
struct ForceWork;
// fw (nullable) with n_force > 0 folds the springs and trap + pair forces into
// the recursion launch as n_force extra blocks.
cudaError_t xdf_launch_forward(const XView& v, cudaStream_t st, ProfMarks* pm, const ForceWork* fw = nullptr,
                               int n_force = 0);
cudaError_t xdf_launch_adjoint(const XView& v, const FinalizeOut& o, cudaStream_t st, ProfMarks* pm);
cudaError_t xdf_launch_vb_value(const XView& v, double* V_out, cudaStream_t st);
