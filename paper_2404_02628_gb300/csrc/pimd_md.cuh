// Ring-polymer springs (a1), trap + Gaussian pair forces (a4), the massive
// Nose-Hoover-chain velocity-Verlet update (a5) and the per-step scalar
// reductions.  Bead arrays are slice-major FP64: x[(j*d + c)*ld + l].
#pragma once
#include "pimd_device.cuh"

struct BeadView {
    int N, P, d, ld;
    double* r;
    double* p;
    double* f;
    double* eta;   // [M][P][d][ld]
    double* peta;
    int M;
};

struct ForceParams {
    double ks;      // spring constant m omega_P^2 = P/beta^2
    double omega2;  // trap omega^2
    double A, inv_s2;
    int mixed;      // FP32 springs and pairs
    int accumulate; // 0: overwrite f, 1: add into f
    double inv_P;   // 1/P (the action weight of V(slice)), formed on the host
    double cpair32; // -2 A / (s^2 sc) for the FP32 pair kernel's scaled coordinates
    float sc32;     // sqrt(log2(e))/s: coordinate scale of the FP32 pair kernel
};

// Fills the derived fields of fp (inv_P, cpair32, sc32) for P beads.  Host only.
void force_constants(ForceParams& fp, int P);

// Double-float constants of the thermostat half step of length tau = dt/2
// ({high, low} floats, formed on the host by nhc_constants).
struct NhcConst {
    float inv_m[2], inv_Q[2], kT[2];
    float ca[2];  // -tau/(4Q): exponent of the chain-link scalings
    float cg[2];  // tau/2: force-update factor
    float ce[2];  // tau/Q: eta drift
    float cp[2];  // -tau/Q: exponent of the momentum scaling
};

struct MDParams {
    double dt, mass, Q, kT;
    double inv_mass, inv_Q;   // 1/mass and 1/Q, formed on the host
    double half_dt, dt_inv_mass;  // dt/2 and dt/mass, formed on the host (nhc_constants)
    int thermostat;
    int nhc_fp32;             // thermostat chain arithmetic in FP32
    float f_inv_mass, f_inv_Q, f_kT, f_half_dt;  // FP32 copies for that mode
    NhcConst nc;                                  // double-float constants (FP64-accurate mode)
};

// Fills mp.nc (and the FP32 copies) from dt, inv_mass, inv_Q, kT.  Host only.
void nhc_constants(MDParams& mp);

// Scalar slots of the per-step reduction (device array of doubles).
enum {
    SC_EINT = 0,   // sum of internal spring energies sum_l E_int^(l)
    SC_GLINK,      // sum_{i<N-1} g(i,i+1) = beta * sum of link spring energies
    SC_L0,         // xi = 0: ln of the diagonal chain product
    SC_LAMBDA,     // ln W_N (forward)
    SC_LAMBDA_B,   // ln W_N (backward)
    SC_U,          // U = sum over slices of (trap + pair) energy
    SC_VIRIAL,     // sum r . grad U
    SC_SPRING_X,   // exchange part of the expected spring energy
    SC_KIN,        // sum p^2/(2m')
    SC_THERMO,     // sum p_eta^2/(2Q) + eta kT
    SC_COUNT
};

// Most particle species with exchange recursions of their own (pimd_set_species).
#define PIMD_MAXSP 4

struct ScalarSources {
    const double* springs; int n_springs;   // [n] E_int partials
    const double* pair; int n_pair;         // [n][2]: energy, virial
    const double* fin; int n_fin;           // [n]
    const double* md; int n_md;             // [n][2]: kinetic, thermostat
    int nsp;                                // species, each with its own exchange recursion
    const double* lsum[PIMD_MAXSP];         // per species: prep partials [n][2]
    int n_lsum[PIMD_MAXSP];
    const double* y_m[PIMD_MAXSP];          // per species: forward Z at index N_s (FP64 path)
    const int* y_e[PIMD_MAXSP];
    const double* c_m[PIMD_MAXSP];          // per species: backward Z at index 0 (FP64 path)
    const int* c_e[PIMD_MAXSP];
    const double* lam[PIMD_MAXSP];          // per species, if set: [2] ln W_N forward/backward (double-float path)
    int N[PIMD_MAXSP];                      // particles per species
    int xi_zero;
    double log_xi;
    double* out;                            // [SC_COUNT]
};

int springs_grid_x(int N);
int pair_grid_x(int N, int pt);   // blocks per slice for pt particles per block
bool pair_block_ok(int pt);       // pt in {64, 128, 256}
constexpr int PAIR_T_MIN = 64;
int md_blocks(int N, int P, int d);

cudaError_t launch_springs(const BeadView& b, const ForceParams& fp, double* f_out, double* part, cudaStream_t st);
cudaError_t launch_pair(const BeadView& b, const ForceParams& fp, double* f_out, double* part, cudaStream_t st, int pt);
cudaError_t launch_md_pre(const BeadView& b, const MDParams& mp, cudaStream_t st);
cudaError_t launch_md_post(const BeadView& b, const MDParams& mp, cudaStream_t st);
cudaError_t launch_md_energy(const BeadView& b, const MDParams& mp, double* part, cudaStream_t st);
cudaError_t launch_scalars(const ScalarSources& s, cudaStream_t st);
cudaError_t launch_zero(double* x, size_t n, cudaStream_t st);
// Seeded initial state: beads ~ N(0, 1) per coordinate, momenta ~ N(0, p_scale^2)
// (p_scale = sqrt(m kT)), padding columns zero.  Counter-based splitmix64
// stream `seed`, two uniforms per coordinate, Box-Muller (cosine branch).
cudaError_t launch_init_state(const BeadView& b, double p_scale, unsigned long long seed, cudaStream_t st);
// Radial bead density of the current configuration added into hist[nbins]:
// bin b = floor(sqrt(r2) / dr) with r2 = x0*x0 + x1*x1 + x2*x2 rounded after
// every operation (no contraction), weight 1 / (N P V_b), V_b the d-dimensional
// shell volume.  nbins <= DENSITY_MAX_BINS.
constexpr int DENSITY_MAX_BINS = 8192;
cudaError_t launch_density(const BeadView& b, int nbins, double dr, double* hist, cudaStream_t st);
// Output i of the splitmix64 stream `seed` (host copy, for per-replica seeds).
unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i);
cudaError_t launch_nonfinite_scan(const double* x, int N, int P, int d, int ld, int* flag, cudaStream_t st);
