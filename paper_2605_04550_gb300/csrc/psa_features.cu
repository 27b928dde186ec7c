// psa_features.cu -- the classifier's inputs (paper Sec. 3.1 and 3.2.1).
//
// Per matrix, one block of 1024 threads reduces the band in FP64 to the
// statistics the global features are built from (norms, symmetry defects,
// diagonal and off-diagonal moduli, the eigenvalue centroid trace(A) / n) and
// samples the symbol f(t) = sum_d abar_d e^{i d t} of the diagonal means abar_d
// at 256 points of [0, 2 pi). For a banded Toeplitz-like matrix of large order
// the symbol curve is where the pseudospectra of the finite sections
// accumulate, so its samples stand in for the eigenvalue set that the paper's
// eigenvalue features use (dense eigenvalues are O(n^3) at n = 20000 and, for
// matrices this far from normal, carry rounding errors of order u * kappa(V)).
// A second kernel turns the statistics and four sigma_min values computed by
// the library's own kernel (z = 0 and the centroid shifted by 0.5, 1, 2) into
// the global feature vector; the per-point kernel writes one BF16 feature row
// per grid point: the Fourier encoding of the normalised coordinates, the
// distances to the centroid and to the symbol curve, the winding number of the
// curve about the point, and the global features.
//
// The paper's own spectrum features are available too: psa_point_set_stats takes
// the statistics over a point set (the eigenvalues of A from a dense eigensolver,
// supplied by the caller), and the per-point kernel runs over any set, as a
// closed polyline (the symbol samples) or as a point set (distance to the
// nearest eigenvalue, Eq. (dist)).
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "psa.h"

namespace psa {
namespace feat {

constexpr int T = PSA_SYMBOL_SAMPLES;
constexpr int kPointFeatures = 33 + PSA_GLOBAL_FEATURES;  // nonzero columns of a feature row
constexpr int NT = 1024;

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];  // same order in every thread
    return s;
}

__device__ __forceinline__ double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = red[0];
    for (int w = 1; w < NT / 32; ++w) s = fmax(s, red[w]);
    return s;
}

__device__ __forceinline__ double block_min(double v, double *red) { return -block_max(-v, red); }

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// stats layout (doubles), see PSA_STAT_* in psa.h
__global__ void __launch_bounds__(NT) k_matrix_stats(const double2 *bands, int n, int kl, int ku, double *stats,
                                                     double2 *symbol)
{
    __shared__ double red[NT / 32];
    __shared__ double2 abar[PSA_MAX_BAND];
    const int W = kl + ku + 1;
    const int tid = threadIdx.x;
    // diagonal means abar_d (d = -kl .. ku), valid rows only
    for (int d = -kl; d <= ku; ++d) {
        double sr = 0.0, si = 0.0;
        const int i0 = d < 0 ? -d : 0, i1 = d > 0 ? n - d : n;
        for (int i = i0 + tid; i < i1; i += NT) {
            const double2 a = bands[(int64_t)(d + kl) * n + i];
            sr += a.x;
            si += a.y;
        }
        sr = block_sum(sr, red);
        si = block_sum(si, red);
        if (tid == 0) abar[d + kl] = make_double2(sr / (double)(i1 - i0), si / (double)(i1 - i0));
    }
    // Frobenius norm, symmetry defects, diagonal and off-diagonal moduli, nonzeros
    double fro = 0.0, asym = 0.0, aherm = 0.0, dsum = 0.0, dsq = 0.0, osum = 0.0, osq = 0.0, nnz = 0.0;
    for (int64_t e = tid; e < (int64_t)W * n; e += NT) {
        const int dk = (int)(e / n), i = (int)(e - (int64_t)dk * n), d = dk - kl, j = i + d;
        if (j < 0 || j >= n) continue;
        const double2 a = bands[e];
        const double m2 = cabs2(a), m = sqrt(m2);
        fro += m2;
        nnz += m > 1e-10 ? 1.0 : 0.0;
        if (d == 0) {
            dsum += m;
            dsq += m2;
        } else {
            osum += m;
            osq += m2;
        }
        // |A_ij - A_ji|^2 and |A_ij - conj(A_ji)|^2 over ordered pairs: a pair whose
        // transpose lies outside the band is met once here and stands for both
        const bool in = (-d >= -kl) && (-d <= ku);
        const double2 b = in ? bands[(int64_t)(-d + kl) * n + j] : make_double2(0.0, 0.0);
        const double wgt = in ? 1.0 : 2.0;
        asym += wgt * ((a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y));
        aherm += wgt * ((a.x - b.x) * (a.x - b.x) + (a.y + b.y) * (a.y + b.y));
    }
    fro = block_sum(fro, red);
    asym = block_sum(asym, red);
    aherm = block_sum(aherm, red);
    dsum = block_sum(dsum, red);
    dsq = block_sum(dsq, red);
    osum = block_sum(osum, red);
    osq = block_sum(osq, red);
    nnz = block_sum(nnz, red);
    // 1-norm (largest column sum) and infinity-norm (largest row sum)
    double cmax = 0.0, rmax = 0.0;
    for (int i = tid; i < n; i += NT) {
        double rs = 0.0, cs = 0.0;
        for (int d = -kl; d <= ku; ++d) {
            if (i + d >= 0 && i + d < n) rs += sqrt(cabs2(bands[(int64_t)(d + kl) * n + i]));
            const int r = i - d;  // column i holds A[i - d][i] = bands[d + kl][i - d]
            if (r >= 0 && r < n) cs += sqrt(cabs2(bands[(int64_t)(d + kl) * n + r]));
        }
        rmax = fmax(rmax, rs);
        cmax = fmax(cmax, cs);
    }
    rmax = block_max(rmax, red);
    cmax = block_max(cmax, red);
    __syncthreads();
    // symbol samples about the centroid
    const double2 cen = abar[kl];
    double sre = 0.0, sim = 0.0, sre2 = 0.0, sim2 = 0.0, rmaxs = 0.0;
    double mnre = INFINITY, mxre = -INFINITY, mnim = INFINITY, mxim = -INFINITY, rmin = INFINITY;
    for (int k = tid; k < T; k += NT) {
        const double t = 2.0 * M_PI * (double)k / (double)T;
        double fr = 0.0, fi = 0.0;
        for (int d = -kl; d <= ku; ++d) {
            double s, c;
            sincos((double)d * t, &s, &c);
            const double2 a = abar[d + kl];
            fr += a.x * c - a.y * s;
            fi += a.x * s + a.y * c;
        }
        symbol[k] = make_double2(fr, fi);
        const double xr = fr - cen.x, xi = fi - cen.y, r = sqrt(xr * xr + xi * xi);
        sre += xr;
        sim += xi;
        sre2 += xr * xr;
        sim2 += xi * xi;
        mnre = fmin(mnre, xr);
        mxre = fmax(mxre, xr);
        mnim = fmin(mnim, xi);
        mxim = fmax(mxim, xi);
        rmaxs = fmax(rmaxs, r);
        rmin = fmin(rmin, r);
    }
    sre = block_sum(sre, red);
    sim = block_sum(sim, red);
    sre2 = block_sum(sre2, red);
    sim2 = block_sum(sim2, red);
    mnre = block_min(mnre, red);
    mxre = block_max(mxre, red);
    mnim = block_min(mnim, red);
    mxim = block_max(mxim, red);
    rmaxs = block_max(rmaxs, red);
    rmin = block_min(rmin, red);
    if (tid == 0) {
        // moduli statistics over the n diagonal and the other in-band positions
        const double nd = (double)n, ndiag = nd;
        const double noff = fmax((double)(W - 1) * nd - (double)(kl * (kl + 1) / 2 + ku * (ku + 1) / 2), 1.0);
        stats[PSA_STAT_CEN_RE] = cen.x;
        stats[PSA_STAT_CEN_IM] = cen.y;
        stats[PSA_STAT_RADIUS] = rmaxs;
        stats[PSA_STAT_FRO] = sqrt(fro);
        stats[PSA_STAT_NORM1] = cmax;
        stats[PSA_STAT_NORMINF] = rmax;
        stats[PSA_STAT_ASYM] = sqrt(asym);
        stats[PSA_STAT_AHERM] = sqrt(aherm);
        stats[PSA_STAT_DIAG_MEAN] = dsum / ndiag;
        stats[PSA_STAT_DIAG_STD] = sqrt(fmax(dsq / ndiag - (dsum / ndiag) * (dsum / ndiag), 0.0));
        stats[PSA_STAT_OFF_MEAN] = osum / noff;
        stats[PSA_STAT_OFF_STD] = sqrt(fmax(osq / noff - (osum / noff) * (osum / noff), 0.0));
        stats[PSA_STAT_NNZ] = nnz;
        stats[PSA_STAT_SYM_RE_MEAN] = sre / T;
        stats[PSA_STAT_SYM_RE_STD] = sqrt(fmax(sre2 / T - (sre / T) * (sre / T), 0.0));
        stats[PSA_STAT_SYM_RE_MIN] = mnre;
        stats[PSA_STAT_SYM_RE_MAX] = mxre;
        stats[PSA_STAT_SYM_IM_MEAN] = sim / T;
        stats[PSA_STAT_SYM_IM_STD] = sqrt(fmax(sim2 / T - (sim / T) * (sim / T), 0.0));
        stats[PSA_STAT_SYM_IM_MIN] = mnim;
        stats[PSA_STAT_SYM_IM_MAX] = mxim;
        stats[PSA_STAT_SYM_RMIN] = rmin;
        stats[PSA_STAT_N] = nd;
        stats[PSA_STAT_BAND] = (double)(kl * 16 + ku);
    }
}

__device__ __forceinline__ float lg(double v) { return (float)log10(fmax(v, 1e-300)); }

// Global feature vector (float32, PSA_GLOBAL_FEATURES): scale-free forms of the
// statistics; sigma4 = sigma_min at z = 0 and at centroid + 0.5, 1, 2.
__global__ void k_global_features(const double *st, const double *sigma4, double eps, float *g)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double R = fmax(st[PSA_STAT_RADIUS], 1e-300);
    const double fro = fmax(st[PSA_STAT_FRO], 1e-300);
    const double n = st[PSA_STAT_N];
    const double rms = fro / sqrt(n);
    const int band = (int)st[PSA_STAT_BAND];
    float v[PSA_GLOBAL_FEATURES] = {};
    v[0] = (float)(st[PSA_STAT_SYM_RE_MEAN] / R);   // f1 .. f8: spectrum stand-in about the centroid
    v[1] = (float)(st[PSA_STAT_SYM_RE_STD] / R);
    v[2] = (float)(st[PSA_STAT_SYM_RE_MIN] / R);
    v[3] = (float)(st[PSA_STAT_SYM_RE_MAX] / R);
    v[4] = (float)(st[PSA_STAT_SYM_IM_MEAN] / R);
    v[5] = (float)(st[PSA_STAT_SYM_IM_STD] / R);
    v[6] = (float)(st[PSA_STAT_SYM_IM_MIN] / R);
    v[7] = (float)(st[PSA_STAT_SYM_IM_MAX] / R);
    v[8] = (float)(st[PSA_STAT_SYM_RMIN] / R);       // f10 (f9 = 1 after scaling)
    v[9] = (float)(st[PSA_STAT_ASYM] / fro);         // f11
    v[10] = (float)(st[PSA_STAT_AHERM] / fro);       // f12
    const double s1 = sqrt(st[PSA_STAT_NORM1] * st[PSA_STAT_NORMINF]);  // bound on sigma_1
    v[11] = lg(s1 / fmax(sigma4[0], 1e-300) + 1e-12);  // f13 with sigma_n = sigma_min at z = 0
    v[12] = (float)(st[PSA_STAT_NORM1] / fro);       // f15
    v[13] = (float)(st[PSA_STAT_NORMINF] / fro);     // f16
    v[14] = (float)(st[PSA_STAT_DIAG_MEAN] / rms);   // f17, f18
    v[15] = (float)(st[PSA_STAT_DIAG_STD] / rms);
    v[16] = (float)(st[PSA_STAT_OFF_MEAN] / rms);    // f19, f20 over the band
    v[17] = (float)(st[PSA_STAT_OFF_STD] / rms);
    v[18] = (float)(st[PSA_STAT_NNZ] / n / 16.0);    // f21 as nonzeros per row
    v[19] = lg(st[PSA_STAT_AHERM] / fro + 1e-12);    // f25
    for (int k = 0; k < 3; ++k) v[20 + k] = lg(R / fmax(sigma4[1 + k], 1e-300));  // f28 .. f30 (exact 2-norm) x R
    v[23] = lg(R);
    v[24] = lg(eps / R);
    v[25] = (float)((band >> 4) / 4.0);
    v[26] = (float)((band & 15) / 8.0);
    v[27] = (float)(log10(n) / 4.0);
    for (int k = 0; k < PSA_GLOBAL_FEATURES; ++k) g[k] = v[k];
}

// Spectrum statistics of a point set (the eigenvalues of A, for the paper's own
// features f1 .. f10 of Sec. 3.1, Table "matrix") about the centroid already in
// stats: they replace the symbol-sample statistics and the radius R.
__global__ void __launch_bounds__(NT) k_point_set_stats(const double2 *pts, int m, double *stats)
{
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;
    const double cx = stats[PSA_STAT_CEN_RE], cy = stats[PSA_STAT_CEN_IM];
    double sre = 0.0, sim = 0.0, sre2 = 0.0, sim2 = 0.0, rmaxs = 0.0;
    double mnre = INFINITY, mxre = -INFINITY, mnim = INFINITY, mxim = -INFINITY, rmin = INFINITY;
    for (int k = tid; k < m; k += NT) {
        const double xr = pts[k].x - cx, xi = pts[k].y - cy, r = sqrt(xr * xr + xi * xi);
        sre += xr;
        sim += xi;
        sre2 += xr * xr;
        sim2 += xi * xi;
        mnre = fmin(mnre, xr);
        mxre = fmax(mxre, xr);
        mnim = fmin(mnim, xi);
        mxim = fmax(mxim, xi);
        rmaxs = fmax(rmaxs, r);
        rmin = fmin(rmin, r);
    }
    sre = block_sum(sre, red);
    sim = block_sum(sim, red);
    sre2 = block_sum(sre2, red);
    sim2 = block_sum(sim2, red);
    mnre = block_min(mnre, red);
    mxre = block_max(mxre, red);
    mnim = block_min(mnim, red);
    mxim = block_max(mxim, red);
    rmaxs = block_max(rmaxs, red);
    rmin = block_min(rmin, red);
    if (tid == 0) {
        const double dm = (double)m;
        stats[PSA_STAT_RADIUS] = rmaxs;
        stats[PSA_STAT_SYM_RE_MEAN] = sre / dm;
        stats[PSA_STAT_SYM_RE_STD] = sqrt(fmax(sre2 / dm - (sre / dm) * (sre / dm), 0.0));
        stats[PSA_STAT_SYM_RE_MIN] = mnre;
        stats[PSA_STAT_SYM_RE_MAX] = mxre;
        stats[PSA_STAT_SYM_IM_MEAN] = sim / dm;
        stats[PSA_STAT_SYM_IM_STD] = sqrt(fmax(sim2 / dm - (sim / dm) * (sim / dm), 0.0));
        stats[PSA_STAT_SYM_IM_MIN] = mnim;
        stats[PSA_STAT_SYM_IM_MAX] = mxim;
        stats[PSA_STAT_SYM_RMIN] = rmin;
    }
}

// points of the curve or set that one shared-memory pass holds
constexpr int kSetChunk = 2048;

// One feature row per point (flat grid index idx[p], or p on the full grid).
// CLOSED: the set is the closed polyline through the symbol samples (distance to the
// polyline, winding number); otherwise a point set such as the eigenvalues (distance
// to the nearest point, no winding number). The set passes through shared memory in
// chunks, each entry preceded by its predecessor on the closed curve.
template <bool CLOSED>
__global__ void k_point_features(double re_min, double im_min, double hx, double hy, int nx, int ny,
                                 const int32_t *idx, int64_t npts, const float *gfeat, const double *st,
                                 const double2 *set, int m, __nv_bfloat16 *x)
{
    __shared__ float2 sh[kSetChunk + 1];
    __shared__ float gf[PSA_GLOBAL_FEATURES];
    const double cr = st[PSA_STAT_CEN_RE], ci = st[PSA_STAT_CEN_IM];
    const float R = (float)fmax(st[PSA_STAT_RADIUS], 1e-30);
    for (int k = threadIdx.x; k < PSA_GLOBAL_FEATURES; k += blockDim.x) gf[k] = gfeat[k];
    const double xc = re_min + 0.5 * hx * (nx - 1), yc = im_min + 0.5 * hy * (ny - 1);
    const double hw = fmax(0.5 * hx * (nx - 1), 1e-300), hh = fmax(0.5 * hy * (ny - 1), 1e-300);
    // every thread of a block takes the same number of passes (the chunk loads need all)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npts; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = base + threadIdx.x;
        const bool live = p < npts;
        const int64_t f = live ? (idx ? (int64_t)idx[p] : p) : 0;
        const int i = (int)(f / nx), j = (int)(f - (int64_t)i * nx);
        const double zr = fma((double)j, hx, re_min), zi = fma((double)i, hy, im_min);
        // distances (about the centroid, in units of R) and winding; for the closed
        // curve dmin is the distance to the polyline through the samples (exact for a
        // curve made of straight pieces, such as the segment of a kl = ku Grcar-type
        // band, whose sensitive zone is a band of width about 2 eps around it)
        const float pr = (float)(zr - cr), pi = (float)(zi - ci);
        float dmin = INFINITY, dsum = 0.f, wind = 0.f;
        for (int c0 = 0; c0 < m; c0 += kSetChunk) {
            const int len = m - c0 < kSetChunk ? m - c0 : kSetChunk;
            __syncthreads();
            for (int k = threadIdx.x; k <= len; k += blockDim.x) {
                const int src = k > 0 ? c0 + k - 1 : (c0 > 0 ? c0 - 1 : m - 1);
                sh[k] = make_float2((float)(set[src].x - cr), (float)(set[src].y - ci));
            }
            __syncthreads();
            if (!live) continue;
            float2 prev = make_float2(sh[0].x - pr, sh[0].y - pi);
            for (int k = 1; k <= len; ++k) {
                const float2 cur = make_float2(sh[k].x - pr, sh[k].y - pi);
                const float dc = sqrtf(cur.x * cur.x + cur.y * cur.y);
                dsum += dc;
                if (CLOSED) {
                    // nearest point of the piece prev -> cur to the point (the origin here)
                    const float ex = cur.x - prev.x, ey = cur.y - prev.y;
                    const float ee = ex * ex + ey * ey;
                    const float t = ee > 0.f ? fminf(fmaxf(-(prev.x * ex + prev.y * ey) / ee, 0.f), 1.f) : 0.f;
                    const float qx = prev.x + t * ex, qy = prev.y + t * ey;
                    dmin = fminf(dmin, sqrtf(qx * qx + qy * qy));
                    // angle swept from prev to cur about the point
                    wind += atan2f(prev.x * cur.y - prev.y * cur.x, prev.x * cur.x + prev.y * cur.y);
                } else {
                    dmin = fminf(dmin, dc);
                }
                prev = cur;
            }
        }
        if (!live) continue;
        float v[64];
        // Fourier encoding of c = (x^, y^) in [-1, 1]^2: [c, sin 2^k c, cos 2^k c], k = 1..6
        const float cx = (float)((zr - xc) / hw), cy = (float)((zi - yc) / hh);
        v[0] = cx;
        v[1] = cy;
#pragma unroll
        for (int k = 1; k <= 6; ++k) {
            const float w = (float)(1 << k);
            float sx, cxx, sy, cyy;
            sincosf(w * cx, &sx, &cxx);
            sincosf(w * cy, &sy, &cyy);
            v[2 + 4 * (k - 1) + 0] = sx;
            v[2 + 4 * (k - 1) + 1] = sy;
            v[2 + 4 * (k - 1) + 2] = cxx;
            v[2 + 4 * (k - 1) + 3] = cyy;
        }
        const float g1 = dmin / R, g3 = dsum / (float)m / R, g2 = sqrtf(pr * pr + pi * pi) / R;
        v[26] = g1;
        v[27] = g2;
        v[28] = g3;
        v[29] = log10f(g1 + 1e-7f);
        v[30] = log10f(g3 + 1e-7f);
        v[31] = CLOSED ? rintf(wind / 6.28318530718f) : 0.f;
        for (int k = 0; k < PSA_GLOBAL_FEATURES; ++k) v[32 + k] = gf[k];
        // the distance to the curve (or set) against the level: log10(dmin / eps), with
        // gf[24] = log10(eps / R)
        v[32 + PSA_GLOBAL_FEATURES] = v[29] - gf[24];
        __nv_bfloat16 *row = x + p * PSA_MLP_IN;
        for (int k = 0; k < kPointFeatures; ++k) row[k] = __float2bfloat16_rn(v[k]);
        for (int k = kPointFeatures; k < PSA_MLP_IN; ++k) row[k] = __float2bfloat16_rn(0.f);
    }
}

// Predicted region (paper Sec. 3.6 and 4): keep[p] = (prob[p] >= tau), then a box
// dilation of radius r on the nx x ny grid.
__global__ void k_region(const float *prob, float tau, int nx, int ny, int r, uint8_t *out)
{
    const int64_t N = (int64_t)nx * ny;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(f / nx), j = (int)(f - (int64_t)i * nx);
        uint8_t hit = 0;
        for (int a = max(i - r, 0); a <= min(i + r, ny - 1) && !hit; ++a)
            for (int b = max(j - r, 0); b <= min(j + r, nx - 1); ++b)
                if (prob[(int64_t)a * nx + b] >= tau) {
                    hit = 1;
                    break;
                }
        out[f] = hit;
    }
}

// slot[key(f)] = f for the points of the region, -1 elsewhere, where key orders
// the grid by 8 x 4 tiles (the work order of the sigma_min kernel's full grid).
__global__ void k_tile_slots(const uint8_t *mask, int nx, int ny, int32_t *slot)
{
    const int tiles_x = (nx + 7) / 8;
    const int64_t S = (int64_t)tiles_x * ((ny + 3) / 4) * 32;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = k >> 5;
        const int lane = (int)(k & 31);
        const int ty = (int)(t / tiles_x), tx = (int)(t - (int64_t)ty * tiles_x);
        const int i = ty * 4 + (lane >> 3), j = tx * 8 + (lane & 7);
        const bool in = i < ny && j < nx && mask[(int64_t)i * nx + j];
        slot[k] = in ? (int32_t)((int64_t)i * nx + j) : -1;
    }
}

}  // namespace feat
}  // namespace psa

using namespace psa::feat;

extern "C" {

int psa_matrix_stats(const psa_band *A, double *stats, psa_c64 *symbol, void *stream)
{
    if (!A || !A->bands || A->n < 1 || A->kl < 0 || A->ku < 0 || A->kl > A->n - 1 || A->ku > A->n - 1 || !stats ||
        !symbol)
        return PSA_EINVAL;
    if (A->kl + A->ku + 1 > PSA_MAX_BAND) return PSA_EUNSUPPORTED;
    k_matrix_stats<<<1, NT, 0, static_cast<cudaStream_t>(stream)>>>(reinterpret_cast<const double2 *>(A->bands), A->n,
                                                                     A->kl, A->ku, stats,
                                                                     reinterpret_cast<double2 *>(symbol));
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

int psa_global_features(const double *stats, const double *sigma4, double eps, float *global, void *stream)
{
    if (!stats || !sigma4 || !global || !(eps > 0.0) || !std::isfinite(eps)) return PSA_EINVAL;
    k_global_features<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(stats, sigma4, eps, global);
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

int psa_point_set_stats(const psa_c64 *set, int32_t m, double *stats, void *stream)
{
    if (!set || !stats || m < 1) return PSA_EINVAL;
    k_point_set_stats<<<1, NT, 0, static_cast<cudaStream_t>(stream)>>>(reinterpret_cast<const double2 *>(set), m,
                                                                        stats);
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

int psa_point_features_set(const psa_grid *g, const int32_t *idx, int64_t n_idx, const double *stats,
                           const psa_c64 *set, int32_t m, int32_t closed, const float *global, uint16_t *x,
                           void *stream)
{
    if (!g || !stats || !set || !global || !x || g->nx < 1 || g->ny < 1 || n_idx < 0 || (n_idx > 0 && !idx) ||
        m < 1 || (closed != 0 && closed != 1))
        return PSA_EINVAL;
    if (!(std::isfinite(g->re_min) && std::isfinite(g->re_max) && std::isfinite(g->im_min) &&
          std::isfinite(g->im_max)) ||
        g->re_min > g->re_max || g->im_min > g->im_max || (int64_t)g->nx * g->ny > 2147483647LL)
        return PSA_EINVAL;
    if (reinterpret_cast<uintptr_t>(x) & 15u) return PSA_EINVAL;
    const int64_t npts = idx ? n_idx : (int64_t)g->nx * g->ny;
    if (npts == 0) return PSA_OK;
    const double hx = g->nx > 1 ? (g->re_max - g->re_min) / (double)(g->nx - 1) : 0.0;
    const double hy = g->ny > 1 ? (g->im_max - g->im_min) / (double)(g->ny - 1) : 0.0;
    const int64_t blocks = (npts + 255) / 256 < 8192 ? (npts + 255) / 256 : 8192;
    const double2 *s = reinterpret_cast<const double2 *>(set);
    __nv_bfloat16 *xb = reinterpret_cast<__nv_bfloat16 *>(x);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (closed)
        k_point_features<true><<<(unsigned)blocks, 256, 0, st>>>(g->re_min, g->im_min, hx, hy, g->nx, g->ny, idx,
                                                                 npts, global, stats, s, m, xb);
    else
        k_point_features<false><<<(unsigned)blocks, 256, 0, st>>>(g->re_min, g->im_min, hx, hy, g->nx, g->ny, idx,
                                                                  npts, global, stats, s, m, xb);
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

int psa_point_features(const psa_grid *g, const int32_t *idx, int64_t n_idx, const double *stats,
                       const psa_c64 *symbol, const float *global, uint16_t *x, void *stream)
{
    return psa_point_features_set(g, idx, n_idx, stats, symbol, PSA_SYMBOL_SAMPLES, 1, global, x, stream);
}

int psa_region(const float *prob, float tau, int32_t nx, int32_t ny, int32_t radius, uint8_t *mask, void *stream)
{
    if (!prob || !mask || nx < 1 || ny < 1 || radius < 0 || radius > 64 || (int64_t)nx * ny > 2147483647LL)
        return PSA_EINVAL;
    const int64_t N = (int64_t)nx * ny;
    const int64_t blocks = (N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192;
    k_region<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(prob, tau, nx, ny, radius, mask);
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

int psa_tile_slots(const uint8_t *mask, int32_t nx, int32_t ny, int32_t *slot, void *stream)
{
    if (!mask || !slot || nx < 1 || ny < 1 || (int64_t)nx * ny > 2147483647LL) return PSA_EINVAL;
    const int64_t S = (int64_t)((nx + 7) / 8) * ((ny + 3) / 4) * 32;
    const int64_t blocks = (S + 255) / 256 < 8192 ? (S + 255) / 256 : 8192;
    k_tile_slots<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(mask, nx, ny, slot);
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

}  // extern "C"
