/*
 * Plain FP64 CPU oracle for bosonic / fictitious-particle PIMD
 * (Xiong, "GPU acceleration of ab initio simulations of large-scale identical
 * particles based on path integral molecular dynamics", arXiv 2404.02628).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Everything is written the slow, literal way, in the paper's order and
 * notation.  Units hbar = m = k_B = 1 (Sec. IV A).  Indices in comments are the
 * paper's 1-based ones; arrays are 0-based.
 *
 * Layout (oracle's own): a configuration r is particle-major,
 *   r[((l-1)*P + (j-1))*d + c]  =  component c of bead j of particle l.
 * Forces use the same layout.
 *
 * Readings of the paper taken here:
 *  - spring constant m*omega_P^2 = P/beta^2           (Sec. III, omega_P = sqrt(P)/(beta hbar))
 *  - forward base case V^[1,0] = 0                     (Sec. III, forward recursion)
 *  - backward base case V^[N+1,N] = 0 (printed "V^[N,N]=0" contradicts the
 *    recursion at u = N)                               (Sec. III, backward recursion)
 *  - 0^0 = 1, so xi = 0 keeps only the k = 1 terms     (Sec. II)
 *  - V(slice) = harmonic trap + Gaussian pairs, both weighted 1/P (Sec. II, Sec. IV B)
 *  - Gaussian width w = s, amplitude A passed in by the caller (Sec. IV B)
 *  - primitive energy estimator PdN/(2 beta) - <spring> + U/P; virial estimator
 *    U/P + (1/2P) sum r.grad U (the paper gives neither formula)
 *  - massive Nose-Hoover chains (Sec. IV A cites them; parameters are not
 *    given): chain length M, Q = kT/omega_P^2, one MTK Trotter half step per side.
 */
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

/* Floating-point type of every quantity.  The oracle is built as written in
 * FP64; the same source built with -DORC_REAL="long double" (type-generic
 * math from <tgmath.h>, nothing else changed) gives an extended-precision
 * twin, used only to measure how far FP64 evaluations -- this oracle's and
 * the GPU's -- sit from the exact result of the same formulas. */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

#define R(r, l, j, c) (r)[(((size_t)(l)) * P + (j)) * d + (c)]

/* |r_a^ja - r_b^jb|^2 */
static real dist2(const real* r, int P, int d, int la, int ja, int lb, int jb)
{
    real s = 0.0;
    for (int c = 0; c < d; ++c) {
        real x = R(r, la, ja, c) - R(r, lb, jb, c);
        s += x * x;
    }
    return s;
}

/* Neumaier-compensated sum of exp(t[i] - m): the plain log-sum-exp of the
 * recursions, made exact to rounding for long sums. */
static real sum_exp_shifted(const real* t, int n, real m)
{
    real s = 0.0, comp = 0.0;
    for (int i = 0; i < n; ++i) {
        real x = exp(t[i] - m);
        real tt = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - tt) + x;
        else comp += (x - tt) + s;
        s = tt;
    }
    return s + comp;
}

static real log_sum_exp(const real* t, int n)
{
    real m = -INFINITY;
    for (int i = 0; i < n; ++i)
        if (t[i] > m) m = t[i];
    if (m == -INFINITY) return -INFINITY;
    return m + log(sum_exp_shifted(t, n, m));
}

/* ln(xi^n) with the convention 0^0 = 1 (Sec. II). */
static real log_xi_pow(real xi, int n)
{
    if (n == 0) return 0.0;
    if (xi == 0.0) return -INFINITY;
    return n * log(xi);
}

/* ------------------------------------------------------------------------ */
/* Cycle energies (Sec. III).                                                */

/* E_int^(v) = 1/2 m omega_P^2 sum_{j=1}^{P-1} (r_v^{j+1} - r_v^j)^2 */
real orc_E_int(int P, int d, const real* r, real beta, int v /* 1-based */)
{
    const real k = P / (beta * beta);
    real s = 0.0;
    for (int j = 0; j < P - 1; ++j) s += dist2(r, P, d, v - 1, j + 1, v - 1, j);
    return 0.5 * k * s;
}

/* All E^[u,v], 1 <= u <= v <= N, by the quadratic iteration of Sec. III:
 *   E^[v,v] = E_int^(v) + 1/2 k (r_v^P - r_v^1)^2
 *   E^[u,v] = E^[u+1,v] - 1/2 k (r_v^P - r_{u+1}^1)^2 + 1/2 k (r_u^P - r_{u+1}^1)^2
 *             + 1/2 k (r_v^P - r_u^1)^2 + E_int^(u)
 * Output E[(u-1)*N + (v-1)]; entries with u > v are left untouched. */
void orc_cycle_energies(int N, int P, int d, const real* r, real beta, real* E)
{
    const real k = P / (beta * beta);
    real* Eint = (real*)malloc(sizeof(real) * (size_t)N);
    for (int v = 1; v <= N; ++v) Eint[v - 1] = orc_E_int(P, d, r, beta, v);
    for (int v = 1; v <= N; ++v) {
        E[(size_t)(v - 1) * N + (v - 1)] =
            Eint[v - 1] + 0.5 * k * dist2(r, P, d, v - 1, P - 1, v - 1, 0);
        for (int u = v - 1; u >= 1; --u) {
            real prev = E[(size_t)u * N + (v - 1)]; /* E^[u+1,v] */
            E[(size_t)(u - 1) * N + (v - 1)] =
                prev - 0.5 * k * dist2(r, P, d, v - 1, P - 1, u, 0)
                + 0.5 * k * dist2(r, P, d, u - 1, P - 1, u, 0)
                + 0.5 * k * dist2(r, P, d, v - 1, P - 1, u - 1, 0) + Eint[u - 1];
        }
    }
    free(Eint);
}

/* ------------------------------------------------------------------------ */
/* Exchange potentials (Sec. III).                                           */

/* Forward recursion, written for every l (the printed one is l = N):
 *   e^{-beta V^[1,l]} = (1/l) sum_{k=1}^{l} xi^{k-1} e^{-beta (E^[l-k+1,l] + V^[1,l-k])}
 * with V^[1,0] = 0.  Output Vf[l] = V^[1,l] for l = 0..N. */
void orc_V_forward(int N, const real* E, real beta, real xi, real* Vf)
{
    real* t = (real*)malloc(sizeof(real) * (size_t)(N + 1));
    Vf[0] = 0.0;
    for (int l = 1; l <= N; ++l) {
        for (int k = 1; k <= l; ++k) {
            real Ec = E[(size_t)(l - k) * N + (l - 1)]; /* E^[l-k+1,l] */
            t[k - 1] = log_xi_pow(xi, k - 1) - beta * (Ec + Vf[l - k]);
        }
        Vf[l] = -(log_sum_exp(t, l) - log((real)l)) / beta;
    }
    free(t);
}

/* Backward recursion:
 *   e^{-beta V^[u,N]} = sum_{l=u}^{N} xi^{l-u} (1/l) e^{-beta (E^[u,l] + V^[l+1,N])}
 * with V^[N+1,N] = 0.  Output Vb[u-1] = V^[u,N] for u = 1..N+1. */
void orc_V_backward(int N, const real* E, real beta, real xi, real* Vb)
{
    real* t = (real*)malloc(sizeof(real) * (size_t)(N + 1));
    Vb[N] = 0.0;
    for (int u = N; u >= 1; --u) {
        int n = 0;
        for (int l = u; l <= N; ++l) {
            real Ec = E[(size_t)(u - 1) * N + (l - 1)]; /* E^[u,l] */
            t[n++] = log_xi_pow(xi, l - u) - log((real)l) - beta * (Ec + Vb[l]);
        }
        Vb[u - 1] = -log_sum_exp(t, n) / beta;
    }
    free(t);
}

/* Connection probabilities (Sec. III), for xi >= 0:
 *   l' <= l : Pr[G(l)=l'] = xi^{l-l'} (1/l) e^{-beta (V^[1,l'-1] + E^[l',l] + V^[l+1,N])} / e^{-beta V^[1,N]}
 *   l' = l+1: Pr[G(l)=l+1] = 1 - e^{-beta (V^[1,l] + V^[l+1,N])} / e^{-beta V^[1,N]}
 *   otherwise 0.
 * Output Pr[(l-1)*(N+1) + (l'-1)] for l = 1..N, l' = 1..N+1. */
void orc_connection_probabilities(int N, const real* E, const real* Vf, const real* Vb,
                                  real beta, real xi, real* Pr)
{
    const real VN = Vf[N];
    for (int l = 1; l <= N; ++l) {
        real* row = Pr + (size_t)(l - 1) * (N + 1);
        for (int lp = 1; lp <= N + 1; ++lp) row[lp - 1] = 0.0;
        for (int lp = 1; lp <= l; ++lp) {
            real Ec = E[(size_t)(lp - 1) * N + (l - 1)]; /* E^[l',l] */
            real lw = log_xi_pow(xi, l - lp) - log((real)l)
                        - beta * (Vf[lp - 1] + Ec + Vb[l]) + beta * VN;
            row[lp - 1] = exp(lw);
        }
        if (l < N) row[l] = 1.0 - exp(-beta * (Vf[l] + Vb[l]) + beta * VN);
    }
}

/* -grad V_xi^[1,N] on every bead (Sec. III):
 *   exterior j=1:  -sum_{l'} Pr[G(l')=l] m w_P^2 (2 r_l^1 - r_l^2 - r_{l'}^P)
 *   exterior j=P:  -sum_{l'} Pr[G(l)=l'] m w_P^2 (2 r_l^P - r_l^{P-1} - r_{l'}^1)
 *   interior:      -m w_P^2 (2 r_l^j - r_l^{j+1} - r_l^{j-1})
 * (l' runs over 1..N; Pr[G(N)=N+1] is zero).  Requires P >= 2.  For P = 2 the
 * two exterior formulas are the whole force. */
void orc_exchange_forces(int N, int P, int d, const real* r, real beta,
                         const real* Pr, real* F)
{
    const real k = P / (beta * beta);
    for (int l = 1; l <= N; ++l) {
        for (int c = 0; c < d; ++c) {
            for (int j = 2; j <= P - 1; ++j)
                R(F, l - 1, j - 1, c) = -k * (2.0 * R(r, l - 1, j - 1, c) - R(r, l - 1, j, c)
                                              - R(r, l - 1, j - 2, c));
            real f1 = 0.0, fP = 0.0;
            for (int lp = 1; lp <= N; ++lp) {
                real p_in = Pr[(size_t)(lp - 1) * (N + 1) + (l - 1)];  /* Pr[G(l')=l] */
                real p_out = Pr[(size_t)(l - 1) * (N + 1) + (lp - 1)]; /* Pr[G(l)=l'] */
                f1 -= p_in * k * (2.0 * R(r, l - 1, 0, c) - R(r, l - 1, 1, c) - R(r, lp - 1, P - 1, c));
                fP -= p_out * k * (2.0 * R(r, l - 1, P - 1, c) - R(r, l - 1, P - 2, c) - R(r, lp - 1, 0, c));
            }
            R(F, l - 1, 0, c) = f1;
            R(F, l - 1, P - 1, c) = fP;
        }
    }
}

/* Expected connected spring energy for the configuration:
 *   sum_l E_int^(l) + sum_{l,l'} Pr[G(l)=l'] 1/2 k (r_l^P - r_{l'}^1)^2
 * which equals -d(beta V_xi)/d(beta) at fixed beads (the primitive estimator's
 * exchange part). */
real orc_spring_expectation(int N, int P, int d, const real* r, real beta, const real* Pr)
{
    const real k = P / (beta * beta);
    real s = 0.0;
    for (int l = 1; l <= N; ++l) s += orc_E_int(P, d, r, beta, l);
    for (int l = 1; l <= N; ++l)
        for (int lp = 1; lp <= N; ++lp) {
            real p = Pr[(size_t)(l - 1) * (N + 1) + (lp - 1)];
            if (p != 0.0) s += p * 0.5 * k * dist2(r, P, d, l - 1, P - 1, lp - 1, 0);
        }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Interaction (Sec. II: U = sum_j V(r_1^j..r_N^j); Sec. IV: trap + Gaussian). */

/* V(slice j) = sum_l 1/2 omega^2 |r_l^j|^2 + 1/2 sum_{i != k} A exp(-|r_i^j - r_k^j|^2 / s^2)
 * Writes U = sum_j V(slice j), F = -grad (U/P) (overwrites), and the virial
 * sum_{l,j} r_l^j . grad_{r_l^j} U. */
void orc_interaction(int N, int P, int d, const real* r, real omega, real A, real s,
                     real* U_out, real* F, real* virial_out)
{
    real U = 0.0, vir = 0.0;
    const real inv_s2 = 1.0 / (s * s);
    for (int j = 0; j < P; ++j) {
        for (int i = 0; i < N; ++i) {
            real g[3] = {0.0, 0.0, 0.0};
            real r2 = 0.0;
            for (int c = 0; c < d; ++c) r2 += R(r, i, j, c) * R(r, i, j, c);
            U += 0.5 * omega * omega * r2;
            for (int c = 0; c < d; ++c) g[c] += omega * omega * R(r, i, j, c);
            for (int kk = 0; kk < N; ++kk) {
                if (kk == i || A == 0.0) continue;
                real q2 = dist2(r, P, d, i, j, kk, j);
                real e = A * exp(-q2 * inv_s2);
                U += 0.5 * e;
                for (int c = 0; c < d; ++c)
                    g[c] += -2.0 * inv_s2 * e * (R(r, i, j, c) - R(r, kk, j, c));
            }
            for (int c = 0; c < d; ++c) {
                R(F, i, j, c) = -g[c] / P;
                vir += R(r, i, j, c) * g[c];
            }
        }
    }
    *U_out = U;
    *virial_out = vir;
}

/* ------------------------------------------------------------------------ */
/* Whole force field for one configuration.                                   */

typedef struct {
    real V_xi;      /* V_xi^[1,N] (forward value)                    */
    real V_xi_bwd;  /* V_xi^[1,N] from the backward recursion         */
    real U_over_P;  /* U/P (trap + pairs)                             */
    real spring;    /* expected connected spring energy               */
    real virial;    /* sum r . grad U                                 */
} orc_force_info;

/* F = -grad(V_xi + U/P).  Returns 0 on success, -1 on bad input / no memory.
 * Pr_out (N*(N+1)) may be NULL. */
int orc_forces(int N, int P, int d, const real* r, real beta, real xi, real omega,
               real A, real s, real* F, orc_force_info* info, real* Pr_out)
{
    if (N < 1 || P < 2 || d < 1 || d > 3 || !(beta > 0.0) || xi < 0.0 || xi > 1.0) return -1;
    real* E = (real*)calloc((size_t)N * N, sizeof(real));
    real* Vf = (real*)malloc(sizeof(real) * (size_t)(N + 1));
    real* Vb = (real*)malloc(sizeof(real) * (size_t)(N + 1));
    real* Pr = Pr_out ? Pr_out : (real*)malloc(sizeof(real) * (size_t)N * (N + 1));
    real* Fi = (real*)malloc(sizeof(real) * (size_t)N * P * d);
    if (!E || !Vf || !Vb || !Pr || !Fi) {
        free(E); free(Vf); free(Vb); if (!Pr_out) free(Pr); free(Fi);
        return -1;
    }
    orc_cycle_energies(N, P, d, r, beta, E);
    orc_V_forward(N, E, beta, xi, Vf);
    orc_V_backward(N, E, beta, xi, Vb);
    orc_connection_probabilities(N, E, Vf, Vb, beta, xi, Pr);
    orc_exchange_forces(N, P, d, r, beta, Pr, F);
    real U, vir;
    orc_interaction(N, P, d, r, omega, A, s, &U, Fi, &vir);
    for (size_t i = 0; i < (size_t)N * P * d; ++i) F[i] += Fi[i];
    if (info) {
        info->V_xi = Vf[N];
        info->V_xi_bwd = Vb[0];
        info->U_over_P = U / P;
        info->spring = orc_spring_expectation(N, P, d, r, beta, Pr);
        info->virial = vir;
    }
    free(E); free(Vf); free(Vb); if (!Pr_out) free(Pr); free(Fi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Molecular dynamics: velocity Verlet with massive Nose-Hoover chains        */
/* (Sec. IV A cites Nose, Hoover, Martyna-Klein-Tuckerman, Jang-Voth).        */

typedef struct {
    real E_prim;     /* PdN/(2 beta) - spring + U/P                          */
    real E_vir;      /* U/P + virial/(2P)                                    */
    real V_xi;
    real U_over_P;
    real kinetic;    /* sum p^2 / (2 m')                                      */
    real spring;
    real H_conserved;/* kinetic + V_xi + U/P + sum (p_eta^2/(2Q) + kT eta)      */
    real virial;
} orc_estimates;

/* One MTK half step of length tau for a single degree of freedom with a chain
 * of M thermostats (positions eta[0..M-1], momenta pe[0..M-1], equal masses Q). */
static void nhc_half(real* p, real m, real* eta, real* pe, int M, real Q, real kT, real tau)
{
    real G;
    G = (M >= 2 ? pe[M - 2] * pe[M - 2] / Q : (*p) * (*p) / m) - kT;
    pe[M - 1] += 0.5 * tau * G;
    for (int k = M - 2; k >= 0; --k) {
        real a = exp(-0.25 * tau * pe[k + 1] / Q);
        G = (k == 0 ? (*p) * (*p) / m : pe[k - 1] * pe[k - 1] / Q) - kT;
        pe[k] = pe[k] * a * a + 0.5 * tau * G * a;
    }
    *p *= exp(-tau * pe[0] / Q);
    for (int k = 0; k < M; ++k) eta[k] += tau * pe[k] / Q;
    for (int k = 0; k <= M - 2; ++k) {
        real a = exp(-0.25 * tau * pe[k + 1] / Q);
        G = (k == 0 ? (*p) * (*p) / m : pe[k - 1] * pe[k - 1] / Q) - kT;
        pe[k] = pe[k] * a * a + 0.5 * tau * G * a;
    }
    G = (M >= 2 ? pe[M - 2] * pe[M - 2] / Q : (*p) * (*p) / m) - kT;
    pe[M - 1] += 0.5 * tau * G;
}

static void fill_estimates(int N, int P, int d, real beta, int M, real Q, real mass,
                           const real* p, const real* eta, const real* pe,
                           const orc_force_info* fi, int thermostat, orc_estimates* est)
{
    const size_t ndof = (size_t)N * P * d;
    real K = 0.0, th = 0.0;
    for (size_t i = 0; i < ndof; ++i) K += 0.5 * p[i] * p[i] / mass;
    if (thermostat)
        for (size_t i = 0; i < ndof * M; ++i) th += 0.5 * pe[i] * pe[i] / Q + eta[i] / beta;
    est->kinetic = K;
    est->V_xi = fi->V_xi;
    est->U_over_P = fi->U_over_P;
    est->spring = fi->spring;
    est->virial = fi->virial;
    est->E_prim = 0.5 * P * d * N / beta - fi->spring + fi->U_over_P;
    est->E_vir = fi->U_over_P + fi->virial / (2.0 * P);
    est->H_conserved = K + fi->V_xi + fi->U_over_P + th;
}

/* Runs nsteps MD steps in place.  State: r, p (N*P*d), eta, peta (N*P*d*M,
 * DOF-major: [dof*M + k]), F = forces of the current r (computed here when
 * *have_forces == 0).  Per step:
 *   NHC(dt/2); p += F dt/2; r += p dt/m'; F = F(r); p += F dt/2; NHC(dt/2).
 * thermostat = 0 runs plain NVE velocity Verlet.  est (nsteps entries, may be
 * NULL) gets the estimators after each step. */
int orc_md_run(int N, int P, int d, real beta, real xi, real omega, real A, real s,
               real dt, int M, real Q, real mass, int thermostat,
               real* r, real* p, real* eta, real* peta, real* F, int* have_forces,
               int nsteps, orc_estimates* est)
{
    const size_t ndof = (size_t)N * P * d;
    const real kT = 1.0 / beta;
    orc_force_info fi;
    if (M < 1) return -1;
    if (!*have_forces) {
        if (orc_forces(N, P, d, r, beta, xi, omega, A, s, F, &fi, NULL)) return -1;
        *have_forces = 1;
    }
    for (int n = 0; n < nsteps; ++n) {
        for (size_t i = 0; i < ndof; ++i) {
            if (thermostat) nhc_half(&p[i], mass, &eta[i * M], &peta[i * M], M, Q, kT, 0.5 * dt);
            p[i] += 0.5 * dt * F[i];
            r[i] += dt * p[i] / mass;
        }
        if (orc_forces(N, P, d, r, beta, xi, omega, A, s, F, &fi, NULL)) return -1;
        for (size_t i = 0; i < ndof; ++i) {
            p[i] += 0.5 * dt * F[i];
            if (thermostat) nhc_half(&p[i], mass, &eta[i * M], &peta[i * M], M, Q, kT, 0.5 * dt);
        }
        if (est) fill_estimates(N, P, d, beta, M, Q, mass, p, eta, peta, &fi, thermostat, &est[n]);
    }
    return 0;
}

/* Estimators of the current state without stepping (forces recomputed). */
int orc_estimators(int N, int P, int d, real beta, real xi, real omega, real A, real s,
                   int M, real Q, real mass, int thermostat, const real* r, const real* p,
                   const real* eta, const real* peta, orc_estimates* est)
{
    orc_force_info fi;
    real* F = (real*)malloc(sizeof(real) * (size_t)N * P * d);
    if (!F) return -1;
    int rc = orc_forces(N, P, d, r, beta, xi, omega, A, s, F, &fi, NULL);
    free(F);
    if (rc) return rc;
    fill_estimates(N, P, d, beta, M, Q, mass, p, eta, peta, &fi, thermostat, est);
    return 0;
}
