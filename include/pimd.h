/*
 * pimd.h -- C ABI of the GB300 bosonic / fictitious-particle PIMD hot path.
 *
 * Method: X. Xiong, "GPU acceleration of ab initio simulations of large-scale
 * identical particles based on path integral molecular dynamics",
 * arXiv 2404.02628.  Units hbar = m = k_B = 1 (Sec. IV A).
 *
 * The library computes, per MD step, for N particles of P beads in d
 * dimensions at inverse temperature beta and exchange parameter xi in [0,1]:
 *   (a1) ring-polymer springs and the spring-energy total     (Sec. III, E_int, E^[v,v])
 *   (a2) the exchange recursions for V_xi^[1,N]                  (Sec. III, forward and
 *                                                                 backward recursions)
 *   (a3) connection probabilities -> endpoint-bead forces       (Sec. III, Pr[G(l)=l'],
 *                                                                 exterior-bead forces)
 *   (a4) harmonic trap + same-slice Gaussian pair forces         (Sec. II U; Sec. IV B)
 *   (a5) velocity Verlet with massive Nose-Hoover chains         (Sec. IV A)
 * The MD samples exp(-beta (V_xi + U/P)) (Sec. II, discretised Z).
 *
 * Conventions for every entry point:
 *  - All device memory belongs to the caller.  Pointers named "device" must
 *    be CUDA device pointers on the current device; the library never calls
 *    cudaMalloc or cudaFree.  Host pointers are plain host memory.
 *  - Work is enqueued on the stream given to pimd_bind / the call and is
 *    asynchronous, except calls that return host data, which synchronise
 *    that stream.
 *  - Errors are returned as pimd_status; no call aborts or throws.  A
 *    human-readable message for the last failure on a handle is available
 *    from pimd_last_error (pimd_global_error for failures before a handle
 *    exists).  Device-side failures (a bounded cross-block wait that gave up)
 *    are recorded in the workspace and reported by the next synchronising
 *    call as PIMD_ETIMEOUT.  Every wait gives up after spin_limit polls; where
 *    a call's configuration leaves spin_limit at 0, or the call takes none
 *    (the exchange-potential calls), the PIMD_SPIN_LIMIT environment variable
 *    (a positive integer, read at each call) sets it, else 2^24.
 *  - Bead arrays are slice-major FP64: element (bead j, component c,
 *    particle l) of an array x lives at x[(j*d + c)*n_pad + l], 0-based,
 *    n_pad >= N a multiple of 32; padding entries are never read.
 *    Thermostat arrays add a leading chain index k: x[((k*P + j)*d + c)*n_pad + l].
 */
#ifndef PIMD_H
#define PIMD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIMD_OK = 0,
    PIMD_EINVAL = 1,      /* bad argument (range, null pointer, size, alignment) */
    PIMD_ENOMEM = 2,      /* caller-provided workspace too small                 */
    PIMD_ECUDA = 3,       /* a CUDA runtime call failed                          */
    PIMD_ETIMEOUT = 4,    /* a bounded cross-block wait gave up on the device    */
    PIMD_ENONFINITE = 5,  /* an energy or force came out NaN/Inf                 */
    PIMD_ESTATE = 6       /* call out of order (e.g. not bound yet)              */
} pimd_status;

enum { PIMD_PREC_FP64 = 0, PIMD_PREC_MIXED = 1 };
/* Gaussian amplitude A in V_pair = A exp(-r^2/s^2): PAPER uses A = g/(pi s^2)
 * as printed in the Hamiltonian of Sec. IV B; RAW uses A = g. */
enum { PIMD_AMP_PAPER = 0, PIMD_AMP_RAW = 1 };
/* Exchange kernel factors exp(-kappa |r_l^P - r_u^1|^2): STORE keeps all
 * N(N+1)/2 of them in the workspace for one step (12 bytes each); RECOMPUTE
 * keeps O(N * 32) and recomputes the rest where they are used. */
enum { PIMD_TABLE_STORE = 0, PIMD_TABLE_RECOMPUTE = 1 };

typedef struct pimd_ctx* pimd_t;

typedef struct {
    double dt;          /* MD time step (default 0.01)                                  */
    int nhc_len;        /* Nose-Hoover chain length M >= 1 (default 4)                  */
    double nhc_Q;       /* thermostat mass; <= 0 selects kT/omega_P^2 = beta/P (default) */
    double mass;        /* bead mass m' of the dynamics (default 1)                     */
    int precision;      /* PIMD_PREC_FP64 (default) or PIMD_PREC_MIXED: springs and pair
                           forces in FP32 (FP64 masters, FP64 accumulation of energies);
                           recursion, probabilities and estimators always FP64          */
    int amp_convention; /* PIMD_AMP_PAPER (default) or PIMD_AMP_RAW                     */
    int table_mode;     /* PIMD_TABLE_STORE (default) or PIMD_TABLE_RECOMPUTE           */
    int thermostat;     /* 1 = massive NHC (default), 0 = plain velocity Verlet (NVE)   */
    int helper_ctas;    /* exchange-recursion helper blocks; 0 = one per SM (default)   */
    int spin_limit;     /* polls before a cross-block wait gives up; 0 = default (2^24,
                           or PIMD_SPIN_LIMIT)                                          */
    int exchange_arith; /* PIMD_XARITH_DF (default): exchange recursion, probabilities and
                           endpoint forces in double-float (FP32 pairs, ~48-bit mantissa, int32
                           exponent) on the FP32 pipe; PIMD_XARITH_FP64: native FP64 throughout */
    int exch_band;      /* look-ahead band width W of the double-float recursion, 2..5
                           (0 = default 4): the chain block adds the W-2 tiles next to the
                           diagonal itself, helper blocks the rest */
    int nhc_fp32;       /* 1: thermostat chain arithmetic in FP32 (state stays FP64, the
                           momentum scaling is applied in FP64); 0: FP64 (default)        */
    int batch_schedule; /* batched replicas only: PIMD_BATCH_PERSISTENT (default 0): the
                           exchange part of a step (prep, factor table, block operators,
                           recursion, band sums of every replica) is one persistent launch
                           working through a dependency-ordered list, beside a grid-stride
                           launch of the springs and pair units on a second stream;
                           PIMD_BATCH_KERNELS: one launch per kernel                      */
} pimd_config;

enum { PIMD_BATCH_PERSISTENT = 0, PIMD_BATCH_KERNELS = 1 };

enum { PIMD_XARITH_DF = 0, PIMD_XARITH_FP64 = 1 };

typedef struct {
    double* r;          /* device, [P][d][n_pad] bead positions                          */
    double* p;          /* device, [P][d][n_pad] momenta                                 */
    double* f;          /* device, [P][d][n_pad] forces -grad(V_xi + U/P), written here  */
    double* eta;        /* device, [M][P][d][n_pad] thermostat positions                 */
    double* peta;       /* device, [M][P][d][n_pad] thermostat momenta                   */
    void* work;         /* device workspace, 256-byte aligned                             */
    size_t work_bytes;  /* its size, at least pimd_workspace_bytes()                      */
    int n_pad;          /* leading dimension of the bead arrays                           */
} pimd_buffers;

/* Per-configuration scalars (Sec. III, Sec. IV; the estimator formulas are
 * not printed in the paper -- see the primitive/virial readings below). */
typedef struct {
    double E_prim;      /* P d N/(2 beta) - spring + U/P                                 */
    double E_vir;       /* U/P + (1/2P) sum_{l,j} r_l^j . grad U                          */
    double V_xi;        /* V_xi^[1,N] from the forward recursion (summed over species)    */
    double U_over_P;    /* (trap + pair energy summed over slices) / P                   */
    double kinetic;     /* sum p^2 / (2 m')                                               */
    double spring;      /* expected connected spring energy sum E_int + sum Pr 1/2 k |dr|^2 */
    double H_conserved; /* kinetic + V_xi + U/P + sum (p_eta^2/(2Q) + eta/beta)           */
    double virial;      /* sum_{l,j} r_l^j . grad U                                       */
    double V_xi_bwd;    /* V_xi^[1,N] from the backward recursion (equals V_xi)           */
    long long step;     /* MD steps taken since pimd_bind / pimd_set_state                */
} pimd_estimates;

/* ---- single system ------------------------------------------------------ */

/* Creates a context for N particles, P >= 2 beads, d in {1,2,3}, beta > 0,
 * trap frequency omega >= 0, Gaussian strength g and width s > 0 (Sec. IV B,
 * width w read as s), xi in [0,1] (Sec. II; 0^0 = 1).  *out receives the
 * handle.  PIMD_EINVAL on a bad argument.  Host only; no GPU work. */
pimd_status pimd_create(int N, int P, int d, double beta, double omega, double g, double s,
                        double xi, pimd_t* out);

/* Several particle species (Sec. II, closing paragraph: the spin-polarised
 * case generalises to coexisting spins, e.g. spin-unpolarised fermions or
 * bosons).  Particles of one species are identical among themselves and
 * distinguishable from the others, so each species gets an exchange
 * potential V_xi of its own over its particles (Sec. III recursions, same
 * beta, P and xi), V_exchange = sum over species; the trap and the Gaussian
 * pair interaction act between all particles alike.  Species s holds the
 * counts[s] consecutive particles after those of species 0..s-1 (so bead
 * arrays keep their layout).  n_species in [1, 4], counts[s] >= 1, sum = N.
 * Call before pimd_workspace_bytes and pimd_bind (PIMD_ESTATE after bind);
 * the default is one species of N.  With several species the springs and
 * pairs run as kernels of their own (not folded into the recursion launch)
 * and the species' recursions run one after another.  Host only. */
pimd_status pimd_set_species(pimd_t ctx, int n_species, const int* counts);

/* Fills *cfg with the defaults listed in pimd_config. */
void pimd_default_config(pimd_config* cfg);

/* Replaces the configuration (before pimd_bind; PIMD_ESTATE after). */
pimd_status pimd_configure(pimd_t ctx, const pimd_config* cfg);

/* Workspace bytes the caller must provide for n_pad (depends on N, P, d, M,
 * table mode and the device's SM count).  Host only. */
pimd_status pimd_workspace_bytes(pimd_t ctx, int n_pad, size_t* bytes);

/* Binds caller-owned device buffers and a CUDA stream (cudaStream_t, may be
 * NULL for the legacy default stream).  Zeroes the thermostat arrays and the
 * step counter; r and p must already hold the initial state.  Computes the
 * forces of r (asynchronously).  Captures the per-step CUDA graph on first
 * pimd_step, so bind before any capture of the caller's own.  The context
 * allocates one small pinned host buffer here (the estimators' read-back),
 * released by pimd_destroy; all device memory stays the caller's. */
pimd_status pimd_bind(pimd_t ctx, const pimd_buffers* bufs, void* stream);

/* Recomputes F = -grad(V_xi + U/P) for the bound r.  If V_total_out (host)
 * is non-NULL, synchronises and stores V_xi + U/P there. */
pimd_status pimd_forces(pimd_t ctx, double* V_total_out);

/* Runs only the exchange part (a1-a3; springs, recursion, probabilities):
 * f_out (device, bead layout) = -grad V_xi.  V_out (host, nullable): V_xi. */
pimd_status pimd_exchange_forces(pimd_t ctx, double* f_out, double* V_out);

/* Runs only the interaction part (a4; trap + pairs): f_out = -grad(U/P),
 * U_out (host, nullable): U/P. */
pimd_status pimd_interaction_forces(pimd_t ctx, double* f_out, double* U_out);

/* Advances nsteps >= 0 MD steps (Sec. IV A; order per step:
 * NHC(dt/2), p += F dt/2, r += p dt/m', forces, p += F dt/2, NHC(dt/2)),
 * replaying one captured CUDA graph per step. */
pimd_status pimd_step(pimd_t ctx, int nsteps);

/* Same step sequence without the CUDA graph (plain launches). */
pimd_status pimd_step_eager(pimd_t ctx, int nsteps);

/* Estimators of the current state (synchronises).  PIMD_ENONFINITE if any
 * field is NaN/Inf, PIMD_ETIMEOUT if a device wait gave up since the last
 * check. */
pimd_status pimd_estimators(pimd_t ctx, pimd_estimates* out);

/* Host blob: a 64-byte header (sizes, step counter) followed by r, p, f,
 * eta, p_eta in the bead layout.  get synchronises; set copies
 * asynchronously from the caller's (ideally pinned) buffer, which must stay
 * valid until the stream reaches the copy.  The forces travel with the state,
 * so a restored run continues bitwise as if uninterrupted. */
pimd_status pimd_state_bytes(pimd_t ctx, size_t* bytes);
pimd_status pimd_get_state(pimd_t ctx, void* host_blob, size_t bytes);
pimd_status pimd_set_state(pimd_t ctx, const void* host_blob, size_t bytes);

/* Radial bead density (Sec. IV B density profiles; per particle, so the
 * ideal gas in its ground state gives exp(-r^2)/pi in d = 2).  For the
 * current configuration, adds rho_b = n_b / (N P V_b) to hist[b] for
 * b < nbins: n_b counts the beads (every particle, every slice) with
 * floor(sqrt(r2) / dr) = b, where dr = r_max / nbins and r2 = x_0^2 + ... +
 * x_{d-1}^2 rounded after every operation (so the bin of each bead is
 * reproducible bit for bit); V_b is the volume of shell b in d dimensions
 * (2 dr; pi (r_{b+1}^2 - r_b^2); 4/3 pi (r_{b+1}^3 - r_b^3)).  Beads at or
 * beyond r_max are not counted.  hist: caller-owned device array of nbins
 * doubles, zeroed by the caller; averaging over calls is the caller's.
 * nbins in [1, 8192].  Stream-ordered, asynchronous. */
pimd_status pimd_density_accumulate(pimd_t ctx, int nbins, double r_max, double* hist);

/* Seeded initial state on the device (Sec. IV: beads drawn from N(0, 1) per
 * coordinate; momenta Maxwell-Boltzmann at kT = 1/beta, i.e. N(0, m/beta)).
 * Generator: splitmix64 (Steele, Lea & Flood, OOPSLA 2014) used counter-wise,
 * output i of stream `seed` = mix(seed + (i + 1) * 0x9E3779B97F4A7C15).
 * Coordinate (q, j, c, l) -- q = 0 beads, 1 momenta; bead j < P, component
 * c < d, particle l < N -- has counter k = ((q P + j) d + c) N + l and uses
 * outputs 2k and 2k + 1 as uniforms u = ((x >> 11) + 1) 2^-53 in (0, 1]:
 * z = sqrt(-2 ln u1) cos(2 pi u2).  Writes r and p of the bound buffers
 * (padding columns zero), zeroes the thermostats and the step counter, and
 * computes the forces of the new r.  Stream-ordered, asynchronous. */
pimd_status pimd_init_state(pimd_t ctx, unsigned long long seed);

/* Runs nsteps MD steps without the graph, with CUDA events between kernels
 * on the bound stream; ms_out[slot] accumulates each kernel's time (slot
 * names from pimd_profile_slot_name).  *n_slots receives the kernel count of
 * one step.  Synchronises.  Used by bench.py for the per-kernel roofline. */
pimd_status pimd_step_profiled(pimd_t ctx, int nsteps, double* ms_out, int max_slots, int* n_slots);
const char* pimd_profile_slot_name(pimd_t ctx, int slot);

/* Autotuner: times the force evaluation (r and p are not advanced) for every
 * candidate launch shape -- the look-ahead band width W of the double-float
 * recursion (those whose workspace fits the bound one), the pair-kernel
 * block of 64, 128 or 256 particles, and (double-float recursion with
 * g != 0) the split of the SMs between recursion helper blocks and force
 * workers that compute springs and trap + pair forces inside the recursion
 * launch, and the number of helper partial sums per block (2, 3 or 4) --
 * and keeps the fastest.  cache_path
 * (nullable): a text file of "device problem|choice" lines; a hit skips the
 * timing, a miss appends the new choice.  The step graph is re-captured on
 * the next pimd_step.  Synchronises. */
pimd_status pimd_autotune(pimd_t ctx, const char* cache_path);
/* The current tuned values (host only).  helpers: recursion helper blocks;
 * force_blocks: force-worker blocks in the recursion launch (0: springs and
 * pairs run as kernels of their own); streams: helper partial sums per block
 * of the double-float recursion (the off-band tiles of a block row or column
 * are dealt to that many helper items, 1..4; default 3).  helpers,
 * force_blocks and streams may be NULL. */
pimd_status pimd_tuning(pimd_t ctx, int* exch_band, int* pair_block, int* helpers, int* force_blocks, int* streams);

/* Debug cross-check (Sec. III, the O(N^3 P) evaluation the paper replaces
 * by its quadratic algorithm): every cycle energy E^[u,v], 1 <= u <= v <= N,
 * of the bound positions straight from its definition -- the springs of the
 * ring made of particles u..v, bead j to j+1 inside each particle, bead P of
 * w to bead 1 of w+1, bead P of v to bead 1 of u, times 1/2 m omega_P^2 =
 * P/(2 beta^2) -- one GPU thread per entry, FP64.  Writes E^[u,v] to
 * E_out[(u-1)*ldE + (v-1)] (device, caller-owned, at least N*ldE doubles);
 * entries with u > v are not written.  ldE >= N, N <= 65535.  Not used by the
 * MD step, whose recursion never forms E.  Stream-ordered, asynchronous. */
pimd_status pimd_cycle_energies_naive(pimd_t ctx, double* E_out, int ldE);

/* Synchronises the bound stream and reports device-side errors. */
pimd_status pimd_sync(pimd_t ctx);

const char* pimd_last_error(pimd_t ctx);
const char* pimd_global_error(void);
void pimd_destroy(pimd_t ctx);

/* ---- batched replicas ----------------------------------------------------- */
/*
 * R independent systems of uneven particle number N_r <= 2047, inverse
 * temperature beta_r and exchange parameter xi_r (for instance the xi and
 * temperature scans of Sec. II's fictitious-particle method), sharing P, d,
 * omega, g, s and one pimd_config.  A step is replayed as one CUDA graph:
 * the thermostat half step, then (batch_schedule = PIMD_BATCH_PERSISTENT)
 * one persistent launch that works through the exchange part of every
 * replica -- prep, factor tiles, block operators, the recursion (one block
 * per replica and direction, longest replicas first), band sums -- in
 * dependency order, while a grid-stride launch on a second stream computes
 * the springs and pair forces; then the endpoint forces and the second half
 * step.  With PIMD_BATCH_KERNELS each part is one launch over all replicas.
 * table_mode, exchange_arith, exch_band and helper_ctas are ignored: the
 * batch always stores the factor table and uses the double-float recursion.
 * nhc_Q <= 0 selects beta_r/P per replica.
 */
typedef struct pimd_batch* pimd_batch_t;

typedef struct {
    double* r;          /* device: replica r's [P][d][n_pad_r] block starts at element
                           offsets[r] (pimd_batch_layout), n_pad_r = N_r rounded up to 32 */
    double* p;          /* device, momenta, same layout                                      */
    double* f;          /* device, forces, same layout (written here)                        */
    double* eta;        /* device, thermostat positions: replica r's [M][P][d][n_pad_r]
                           block at M * offsets[r]                                           */
    double* peta;       /* device, thermostat momenta, same layout as eta                    */
    void* work;         /* device workspace, 256-byte aligned                                */
    size_t work_bytes;  /* its size, at least pimd_batch_workspace_bytes()                   */
} pimd_batch_buffers;

/* N, beta, xi: host arrays of R entries (N_r in [1, 2047], beta_r > 0,
 * xi_r in [0,1]).  Host only. */
pimd_status pimd_batch_create(int R, const int* N, int P, int d, const double* beta, const double* xi,
                              double omega, double g, double s, pimd_batch_t* out);
pimd_status pimd_batch_configure(pimd_batch_t b, const pimd_config* cfg);
/* offsets: host array of R + 1 entries; offsets[R] = total elements per bead array. */
pimd_status pimd_batch_layout(pimd_batch_t b, size_t* offsets);
pimd_status pimd_batch_workspace_bytes(pimd_batch_t b, size_t* bytes);
/* As pimd_bind: zeroes the thermostats and the step counter and computes the
 * forces of r; r and p must hold the initial state. */
pimd_status pimd_batch_bind(pimd_batch_t b, const pimd_batch_buffers* bufs, void* stream);
pimd_status pimd_batch_forces(pimd_batch_t b);
/* As pimd_init_state for every replica; replica r uses the stream whose seed
 * is output r of the splitmix64 stream `seed`. */
pimd_status pimd_batch_init_state(pimd_batch_t b, unsigned long long seed);
/* Captures one batched step as a CUDA graph on a private stream (done by the
 * first pimd_batch_step otherwise). */
pimd_status pimd_batch_capture_graph(pimd_batch_t b);
pimd_status pimd_batch_step(pimd_batch_t b, int nsteps);
pimd_status pimd_batch_step_eager(pimd_batch_t b, int nsteps);
pimd_status pimd_batch_step_profiled(pimd_batch_t b, int nsteps, double* ms_out, int max_slots, int* n_slots);
const char* pimd_batch_profile_slot_name(pimd_batch_t b, int slot);
/* out: host array of R estimates (synchronises). */
pimd_status pimd_batch_estimators(pimd_batch_t b, pimd_estimates* out);
/* Autotuner of the batched step (as pimd_autotune): the pair block of 64, 128
 * or 256 particles and the schedule (persistent or one launch per kernel),
 * cached by device and (R, sum N, sum N^2, P, d). */
pimd_status pimd_batch_autotune(pimd_batch_t b, const char* cache_path);
/* The batch's current pair-kernel block (host only; any time after create). */
pimd_status pimd_batch_tuning(pimd_batch_t b, int* pair_block);
/* The batch's current schedule, PIMD_BATCH_PERSISTENT or PIMD_BATCH_KERNELS
 * (host only; the autotuner may change it). */
pimd_status pimd_batch_schedule(pimd_batch_t b, int* schedule);
pimd_status pimd_batch_sync(pimd_batch_t b);
const char* pimd_batch_last_error(pimd_batch_t b);
void pimd_batch_destroy(pimd_batch_t b);

/* ---- exchange potential alone (for autograd) --------------------------- */
/*
 * V_ends(r^1, r^P) = V_xi^[1,N] - sum_l E_int^(l): the part of the exchange
 * potential (Sec. III) that depends on the endpoint beads only, for spring
 * constant k = P/beta^2 (so the caller supplies P).  r1 and rP are device
 * arrays [d][ld] (component c of particle l at c*ld + l), ld >= N.
 */
typedef struct pimd_vb* pimd_vb_t;

/* The handle computes with the double-float recursion.  Its factor table is
 * stored up to N = 16383 and recomputed where used above (so N = 40000 needs
 * O(32 N) workspace instead of 12 N^2 / 2 bytes); pimd_vb_set_table_mode
 * overrides that (PIMD_TABLE_STORE, PIMD_TABLE_RECOMPUTE, or -1 for the
 * automatic choice) and changes pimd_vb_workspace_bytes accordingly. */
pimd_status pimd_vb_create(int N, int P, int d, double beta, double xi, pimd_vb_t* out);
pimd_status pimd_vb_set_table_mode(pimd_vb_t h, int table_mode);
pimd_status pimd_vb_workspace_bytes(pimd_vb_t h, size_t* bytes);
/* V_out: device double.  Saves the recursion state in work for backward. */
pimd_status pimd_vb_forward(pimd_vb_t h, const double* r1, const double* rP, int ld,
                            void* work, size_t work_bytes, double* V_out, void* stream);
/* Adjoint (Sec. III connection probabilities): g_r1 = gV * dV_ends/dr^1 and
 * g_rP = gV * dV_ends/dr^P ([d][ld], overwritten).  gV: device double.
 * Must follow pimd_vb_forward on the same arrays and workspace. */
pimd_status pimd_vb_backward(pimd_vb_t h, const double* r1, const double* rP, int ld,
                             void* work, size_t work_bytes, const double* gV,
                             double* g_r1, double* g_rP, void* stream);
/* Synchronises `stream` and reports device-side failures of the earlier
 * pimd_vb_forward / pimd_vb_backward calls on this workspace: PIMD_ETIMEOUT
 * if a bounded cross-block wait of the recursion gave up (the error word in
 * the workspace is then cleared, so the next forward starts clean), PIMD_OK
 * otherwise.  A forward whose wait gave up writes NaN to V_out, and a
 * backward after it writes NaN gradients, so callers that cannot synchronise
 * still see invalid results.  work, work_bytes: as given to the calls. */
pimd_status pimd_vb_sync(pimd_vb_t h, void* work, size_t work_bytes, void* stream);
void pimd_vb_destroy(pimd_vb_t h);

/* Same value as pimd_vb_forward (V_ends), for callers that cannot allocate
 * device memory: a host program or plug-in that only receives the input and
 * output arrays from another code (for instance an MD engine that owns the
 * device heap, or a caller inside a region where allocation is not allowed)
 * and so cannot provide the workspace pimd_vb_forward needs.  The paper has
 * no counterpart; this is a packaging variant of the forward recursion.
 *
 * Scratch lives in a fixed 8 MiB array inside the library, which every GPU
 * that loads the library keeps until the process exits.  N must be at most
 * 1024, otherwise PIMD_EINVAL with a message; no cudaMalloc/cudaFree or other
 * allocating routine is called.  r1, rP: device [d][ld]; V_out: device double.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current), so make that first call before any
 * stream capture.  All calls share the one array and each call overwrites it:
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads) race and give wrong results; serialise them on one stream.
 * If a bounded wait of the recursion gives up (see PIMD_SPIN_LIMIT), the
 * call still returns PIMD_OK (it does not synchronise) but writes NaN to
 * *V_out, so the failure shows in the result itself. */
pimd_status pimd_vb_forward_noalloc(int N, int P, int d, double beta, double xi, const double* r1,
                                    const double* rP, int ld, double* V_out, void* stream);

/* ---- measurement probes (roofline denominators) ------------------------------ */
/* The paper has no counterpart: these calls measure, on the current device,
 * what bounds the hot path's kernels, for the roofline fractions that
 * bench.py reports. */
typedef struct {
    double fp64_tflops;  /* FP64 FMA throughput, 2 flops per FMA                       */
    double fp32_tflops;  /* FP32 FMA throughput, 2 flops per FMA                       */
    double ex2_per_s;    /* MUFU ex2.approx.f32 results per second (whole device)     */
    int sms;             /* streaming multiprocessors                                  */
} pimd_rates;
/* Runs three throughput kernels (eight independent FMA / ex2 chains per
 * thread, four 256-thread blocks per SM, a warm-up launch then one timed
 * launch each, CUDA events) and fills *out.  sink: caller-owned device
 * buffer of at least 8 bytes (never written in practice; keeps the
 * arithmetic alive).  Synchronises the stream.  Takes about 0.1 s. */
pimd_status pimd_probe_rates(double* sink, pimd_rates* out, void* stream);

/* Latency of the recursion chain's dependent core (Sec. III forward
 * recursion in the factorised form y_J = Q_J y_{J-1} + G_J s_J): one
 * 256-thread block iterates y_it = Q_k y_{it-1} + G_k s, k = it mod nblk, for
 * n_iter iterations with the chain's own double-float segment products
 * (split warps per tile, 32/split columns each; split in {1, 2, 4}), warp-0
 * sum and two named barriers per iteration, everything in shared memory.
 * Q, G: device, nblk row-major 32x32 FP64 tiles (entries >= 0); y0, s:
 * device, 32 entries >= 0; nblk in [1, 8].  Writes the final iterate to
 * y_out (device, 32 doubles; numerically the product the chain computes) and
 * the clock64 cycles of the iteration loop to *cycles (device).
 * Stream-ordered, asynchronous. */
pimd_status pimd_probe_chain(int nblk, int n_iter, int split, const double* Q, const double* G, const double* y0,
                             const double* s, double* y_out, long long* cycles, void* stream);

/* ---- xi extrapolation (host only) ------------------------------------------ */
/*
 * Fictitious-particle thermodynamics (Sec. I and Sec. IV D): an observable is
 * simulated at xi in [0, 1], where exp(-beta (V_xi + U/P)) is a probability
 * density, and carried to the fermionic value xi = -1 by a fit in xi.  The
 * paper does not print the fitting form; this call fits a polynomial of the
 * given degree (2: the quadratic form of the xi-extrapolation literature the
 * paper cites) by weighted least squares, weights 1/sigma_i^2, and evaluates it
 * at xi_target.
 *   n points (xi[i], E[i], sigma[i] > 0), n >= degree + 1, 0 <= degree <= 6;
 *   *value: the fitted polynomial at xi_target; *value_sigma (nullable): its
 *   standard error from the parameters' covariance; *chi2 (nullable): the
 *   weighted residual sum of squares; coef (nullable, degree + 1 entries):
 *   coefficients in powers of xi, constant term first.
 * PIMD_EINVAL on bad input or when the points do not determine the
 * polynomial (fewer distinct xi than degree + 1).  Host only; no GPU work. */
pimd_status pimd_xi_extrapolate(int n, const double* xi, const double* E, const double* sigma, int degree,
                                double xi_target, double* value, double* value_sigma, double* chi2, double* coef);

#ifdef __cplusplus
}
#endif
#endif /* PIMD_H */
