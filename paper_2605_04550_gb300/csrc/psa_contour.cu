// psa_contour.cu -- the bracketed Newton iteration that refines eps-contour crossings
// along grid rows: the level set sigma_min(zI - A) = eps of paper Sec. 2 (Definition
// "Pseudospectrum") on the grid lines of Sec. 2.1. A crossing of row i lies between
// columns j and j+1 where sigma - eps changes sign; Newton's method on
// f(x) = sigma(x + i y_i) - eps with f'(x) = d sigma / d Re z (psa_sigma_min_grad)
// is kept inside the shrinking bracket, and a step that leaves it (or a slope of no
// use) is replaced by bisection. The evaluations are psa_sigma_min_grad calls; these
// kernels hold the rest of the iteration's arithmetic, so the host only launches.
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "psa.h"

namespace psa {
namespace {

__device__ __forceinline__ double grid_x(const psa_grid &g, int j)
{
    const double h = g.nx > 1 ? (g.re_max - g.re_min) / (double)(g.nx - 1) : 0.0;
    return fma((double)j, h, g.re_min);
}

__device__ __forceinline__ double grid_y(const psa_grid &g, int i)
{
    const double h = g.ny > 1 ? (g.im_max - g.im_min) / (double)(g.ny - 1) : 0.0;
    return fma((double)i, h, g.im_min);
}

// Bracket [x_j, x_{j+1}] of each crossing, its row's ordinate, the sign of f at the
// left end, and the first iterate: the interpolation of log sigma between the bracket
// ends, kept within [0.05, 0.95] of the bracket (the midpoint when undefined).
__global__ void k_contour_init(int m, const int32_t *rows, const int32_t *cols, psa_grid g, const double *s_lo,
                               const double *s_hi, double eps, double *x, double *lo, double *hi, double *y,
                               uint8_t *flo_neg, uint8_t *done, double *resid, double2 *z)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const double a = grid_x(g, cols[c]), b = grid_x(g, cols[c] + 1), yy = grid_y(g, rows[c]);
        const double la = log(fmax(s_lo[c], 1e-300)), lb = log(fmax(s_hi[c], 1e-300));
        double t = (log(eps) - la) / (lb - la);
        t = isfinite(t) ? fmin(fmax(t, 0.05), 0.95) : 0.5;
        const double x0 = a + t * (b - a);
        lo[c] = a;
        hi[c] = b;
        y[c] = yy;
        x[c] = x0;
        flo_neg[c] = s_lo[c] <= eps ? 1 : 0;
        done[c] = 0;
        resid[c] = INFINITY;
        z[c] = make_double2(x0, yy);
    }
}

// One iteration for the crossings idx[0 .. na) that are still running, given sigma and
// grad_z = d sigma / d Re z + i d sigma / d Im z at their current iterates.
__global__ void k_contour_step(int na, const int32_t *idx, const double *sigma, const double2 *grad_z, double eps,
                               double rtol, double *x, double *lo, double *hi, const double *y,
                               const uint8_t *flo_neg, uint8_t *done, double *resid, double2 *z)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
        const int c = idx[a];
        const double f = sigma[a] - eps, slope = grad_z[a].x;
        const double r = fabs(f) / eps;
        resid[c] = r;
        const bool conv = r <= rtol;
        // the bracket end with the sign f had at the left grid point moves to x
        const bool same_as_lo = (f <= 0.0) == (flo_neg[c] != 0);
        const double xc = x[c];
        const double l = same_as_lo ? xc : lo[c], h = same_as_lo ? hi[c] : xc;
        lo[c] = l;
        hi[c] = h;
        double xn = xc - f / slope;
        if (!(isfinite(xn) && xn > l && xn < h)) xn = 0.5 * (l + h);
        const bool narrow = h - l <= 4e-16 * fmax(fabs(l), 1.0);
        if (conv || narrow) done[c] = 1;
        if (!conv) x[c] = xn;
        z[c] = make_double2(conv ? xc : xn, y[c]);
    }
}

unsigned blocks_for(int m) { return (unsigned)((m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024); }

}  // namespace
}  // namespace psa

using namespace psa;

extern "C" {

int psa_contour_init(int32_t m, const int32_t *rows, const int32_t *cols, const psa_grid *g, const double *s_lo,
                     const double *s_hi, double eps, double *x, double *lo, double *hi, double *y, uint8_t *flo_neg,
                     uint8_t *done, double *resid, psa_c64 *z, void *stream)
{
    if (m < 0 || !g || g->nx < 2 || g->ny < 1 || !(eps > 0.0) || !std::isfinite(eps)) return PSA_EINVAL;
    if (m == 0) return PSA_OK;
    if (!rows || !cols || !s_lo || !s_hi || !x || !lo || !hi || !y || !flo_neg || !done || !resid || !z)
        return PSA_EINVAL;
    k_contour_init<<<blocks_for(m), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        m, rows, cols, *g, s_lo, s_hi, eps, x, lo, hi, y, flo_neg, done, resid, reinterpret_cast<double2 *>(z));
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

int psa_contour_step(int32_t na, const int32_t *idx, const double *sigma, const psa_c64 *grad_z, double eps,
                     double rtol, double *x, double *lo, double *hi, const double *y, const uint8_t *flo_neg,
                     uint8_t *done, double *resid, psa_c64 *z, void *stream)
{
    if (na < 0 || !(eps > 0.0) || !std::isfinite(eps) || !(rtol >= 0.0)) return PSA_EINVAL;
    if (na == 0) return PSA_OK;
    if (!idx || !sigma || !grad_z || !x || !lo || !hi || !y || !flo_neg || !done || !resid || !z) return PSA_EINVAL;
    k_contour_step<<<blocks_for(na), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        na, idx, sigma, reinterpret_cast<const double2 *>(grad_z), eps, rtol, x, lo, hi, y, flo_neg, done, resid,
        reinterpret_cast<double2 *>(z));
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

}  // extern "C"
