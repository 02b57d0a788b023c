// Extrapolation of fictitious-particle energies in xi (arXiv 2404.02628,
// Sec. I and Sec. IV D: results for xi in [0, 1], where the path-integral
// weight is non-negative, carried to the fermionic value xi = -1).  Host
// arithmetic only: a weighted least-squares polynomial in xi, solved by a
// Cholesky factorisation of the normal equations in the scaled variable
// t = (xi - mean) / spread, and the value and variance of the polynomial at
// the target point from the parameters' covariance.
#include <math.h>
#include <string.h>

#include "../../include/pimd.h"

namespace {
constexpr int XI_MAXDEG = 6;

// In-place Cholesky factor L (lower) of the n x n SPD matrix A; false if not SPD.
bool cholesky(double* A, int n)
{
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return false;
        const double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    return true;
}

// Solves L L^T x = b in place.
void chol_solve(const double* L, int n, double* b)
{
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i * n + k] * b[k];
        b[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = b[i];
        for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * b[k];
        b[i] = t / L[i * n + i];
    }
}
}  // namespace

extern "C" pimd_status pimd_xi_extrapolate(int n, const double* xi, const double* E, const double* sigma, int degree,
                                           double xi_target, double* value, double* value_sigma, double* chi2,
                                           double* coef)
{
    if (n < 1 || !xi || !E || !sigma || !value || degree < 0 || degree > XI_MAXDEG || n < degree + 1)
        return PIMD_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!(sigma[i] > 0.0) || !isfinite(E[i]) || !isfinite(xi[i])) return PIMD_EINVAL;
    const int m = degree + 1;
    double lo = xi[0], hi = xi[0], mean = 0.0;
    for (int i = 0; i < n; ++i) {
        lo = fmin(lo, xi[i]);
        hi = fmax(hi, xi[i]);
        mean += xi[i];
    }
    mean /= n;
    const double spread = (hi > lo) ? 0.5 * (hi - lo) : 1.0;
    double A[XI_MAXDEG + 1][XI_MAXDEG + 1], b[XI_MAXDEG + 1];
    memset(A, 0, sizeof A);
    memset(b, 0, sizeof b);
    for (int i = 0; i < n; ++i) {
        const double t = (xi[i] - mean) / spread, w = 1.0 / (sigma[i] * sigma[i]);
        double pj = 1.0;
        double pw[XI_MAXDEG + 1];
        for (int j = 0; j < m; ++j) {
            pw[j] = pj;
            pj *= t;
        }
        for (int j = 0; j < m; ++j) {
            b[j] += w * pw[j] * E[i];
            for (int k = 0; k <= j; ++k) A[j][k] += w * pw[j] * pw[k];
        }
    }
    double L[(XI_MAXDEG + 1) * (XI_MAXDEG + 1)];
    for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k) L[j * m + k] = (k <= j) ? A[j][k] : A[k][j];
    if (!cholesky(L, m)) return PIMD_EINVAL;  // too few distinct xi for the degree
    double c[XI_MAXDEG + 1];
    for (int j = 0; j < m; ++j) c[j] = b[j];
    chol_solve(L, m, c);  // coefficients in t
    // value and variance at the target: v = sum_j c_j t0^j, var = p^T (A^-1) p
    const double t0 = (xi_target - mean) / spread;
    double p[XI_MAXDEG + 1], q[XI_MAXDEG + 1], pj = 1.0, v = 0.0;
    for (int j = 0; j < m; ++j) {
        p[j] = q[j] = pj;
        v += c[j] * pj;
        pj *= t0;
    }
    chol_solve(L, m, q);
    double var = 0.0;
    for (int j = 0; j < m; ++j) var += p[j] * q[j];
    *value = v;
    if (value_sigma) *value_sigma = sqrt(fmax(var, 0.0));
    if (chi2) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const double t = (xi[i] - mean) / spread;
            double f = 0.0, tj = 1.0;
            for (int j = 0; j < m; ++j) {
                f += c[j] * tj;
                tj *= t;
            }
            const double r = (E[i] - f) / sigma[i];
            s += r * r;
        }
        *chi2 = s;
    }
    if (coef) {
        // back to powers of xi: t^j = ((xi - mean)/spread)^j expanded binomially
        double out[XI_MAXDEG + 1] = {0.0};
        for (int j = 0; j < m; ++j) {
            const double cj = c[j] / pow(spread, j);
            double binom = 1.0;  // C(j, k)
            for (int k = 0; k <= j; ++k) {
                out[k] += cj * binom * pow(-mean, j - k);
                binom = binom * (j - k) / (k + 1);
            }
        }
        for (int j = 0; j < m; ++j) coef[j] = out[j];
    }
    return PIMD_OK;
}
