// Exchange part of the PIMD force field (arXiv 2404.02628, Sec. III): the
// forward and backward recursions for V_xi^[1,N], the connection
// probabilities, and the endpoint-bead forces they give.
//
// Factorised form used on the GPU.  With a_i = r_i^P, b_k = r_k^1 (0-based
// particles), kappa = m P / (2 beta hbar^2) and g(i,k) = kappa |a_i - b_k|^2,
// every cycle energy of Sec. III splits as
//   beta E^[u,v] = beta (C'_v - C_{u-1}) + g(v,u),
// where C is the prefix of (E_int + inter-particle link) energies.  The prefix
// cancels from every ratio the method uses, which leaves only the endpoint
// Gaussians K[i][k] = exp(-g(i,k)) and the per-particle factor
//   rho[i] = exp(g(i,i+1)) / ((i+1) xi)   (i < N-1),   rho[N-1] = 1/(N xi).
// The forward recursion of Sec. III becomes the triangular solve
//   y[0] = 1,    y[i+1] = rho[i] * sum_{k<=i} K[i][k] y[k],
// the backward recursion its transpose
//   c[N] = 1,    c[k] = sum_{i>=k} K[i][k] rho[i] c[i+1],
// with Z = y[N] = c[0],  V_xi = sum E_int + sum link - (N ln xi + ln Z)/beta,
// and the connection probabilities are
//   Pr[G(i)=k]   = K[i][k] y[k] z[i] / Z   (k <= i),  z[i] = rho[i] c[i+1],
//   Pr[G(i)=i+1] = 1 - y[i+1] c[i+1] / Z.
// The endpoint forces need only the row sums sum_k K y (1, b_k) (forward) and
// the column sums sum_i K z (1, a_i) (backward): the backward recursion is the
// adjoint of the forward one, so no separate O(N^2) probability pass exists.
#pragma once
#include "pimd_device.cuh"

#define EX_THREADS 256
#define EX_WARPS 8
#define EX_LD 33  // padded leading dimension of a staged tile

struct ExchView {
    int N, nb, d, S;        // particles, 32-blocks, dimension, helper streams per block
    int store;              // 1: all tiles stored; 0: only diagonal + subdiagonal tiles
    int xi_zero;            // xi == 0: no exchange (Pr = identity)
    double kappa, ks, beta, log_xi;
    const double* a;        // bead P: component c of particle i at a[c*lda + i]
    const double* b;        // bead 1
    int lda, ldb;
    double* Km; int* Ke;    // tiles [tile][k][i] (1024 each)
    double* rho_m; int* rho_e;   // [nb*32]
    double* y_m; int* y_e;       // [nb*32 + 1]
    double* c_m; int* c_e;       // [nb*32 + 1]
    double* z_m; int* z_e;       // [nb*32]
    double* part_m; int* part_e; // helper partials [2][nb][S][32] x 4 doubles / 1 int
    double* band_m; int* band_e; // band partials [2][nb][2][32] x 4 doubles / 1 int
    int* flags;                  // [2][nb] chain flags, then [2][nb][S] partial flags
    int* err;
    int spin_limit;
    int n_help_f, n_help_b;
    double* lsum;                // prep partial sums [gridDim][2]: link energy, xi=0 log terms
};

__host__ __device__ inline long long ex_tile_index(const ExchView& v, int J, int I)
{
    if (v.store) return (long long)J * (J + 1) / 2 + I;
    return (J == I) ? (long long)J : (long long)v.nb + J - 1;  // band: diag then subdiag
}

// Launch helpers (implemented in pimd_exchange.cu).
struct FinalizeOut {
    double* f;             // force array [P][d][n_pad] or null
    int ldf, P;            // leading dimension (n_pad) and bead count
    double* g1; double* gP;// gradient mode: dV/dr^1, dV/dr^P ([d][ld]); null otherwise
    int ldg;
    const double* gscale;  // gradient mode: device scalar multiplying the gradient
    double* part;          // per-block partial sums [grid][1]: exchange spring energy
};

// Optional per-kernel event marks (bench profiling); null = no marks.
struct ProfMarks {
    cudaEvent_t ev[64];
    const char* name[64];
    int n;
};
void prof_mark(ProfMarks* pm, const char* name, cudaStream_t st);

cudaError_t exch_launch_forward(const ExchView& v, cudaStream_t st, int coop, ProfMarks* pm = nullptr);
cudaError_t exch_launch_adjoint(const ExchView& v, const FinalizeOut& o, int nblk_fin, cudaStream_t st,
                                ProfMarks* pm = nullptr);
cudaError_t exch_launch_vb_value(const ExchView& v, int nprep, double* V_out, cudaStream_t st);
int exch_prep_blocks(int N);
int exch_finalize_blocks(int N);
size_t exch_recursion_smem();
