// Debug cross-check of the cycle energies (arXiv 2404.02628, Sec. III): every
// E^[u,v] straight from its definition, one thread per entry -- the
// O(N^3 P) evaluation the paper describes before its quadratic algorithm.
// The hot path never forms E (its factorised recursion only needs row
// constants); this mode exists to check them against an independent route.
#include "pimd_md.cuh"

namespace {

// E^[u,v] = 1/2 k sum over the springs of the ring of particles u..v (0-based
// here): bead j -> j+1 inside each particle w, bead P of w -> bead 1 of w+1
// for w < v, and bead P of v -> bead 1 of u.  FP64, accumulated particle by
// particle in ring order.
__global__ void __launch_bounds__(256) cycle_naive_kernel(BeadView b, double half_k, double* E, int ldE)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int u = blockIdx.y;
    if (v >= b.N || v < u) return;
    const size_t sd = (size_t)b.d * b.ld;  // stride of one slice
    double s = 0.0;
    for (int w = u; w <= v; ++w) {
        const int nxt = (w < v) ? w + 1 : u;
        for (int c = 0; c < b.d; ++c) {
            const double* x = b.r + (size_t)c * b.ld;
            for (int j = 0; j + 1 < b.P; ++j) {
                const double dx = x[(size_t)(j + 1) * sd + w] - x[(size_t)j * sd + w];
                s = fma(dx, dx, s);
            }
            const double dl = x[nxt] - x[(size_t)(b.P - 1) * sd + w];
            s = fma(dl, dl, s);
        }
    }
    E[(size_t)u * ldE + v] = half_k * s;
}

}  // namespace

cudaError_t launch_cycle_naive(const BeadView& b, double ks, double* E, int ldE, cudaStream_t st)
{
    if (b.N < 1 || b.N > 65535) return cudaErrorInvalidValue;
    const dim3 grid((b.N + 255) / 256, b.N);
    cycle_naive_kernel<<<grid, 256, 0, st>>>(b, 0.5 * ks, E, ldE);
    return cudaGetLastError();
}
