// psa_grad.cuh -- sigma_min(zI - A) with its adjoint gradients at explicit points z.
//
// For a simple smallest singular value sigma of B = zI - A with left and right
// singular vectors u, v (B v = sigma u, B^* u = sigma v), first-order perturbation
// gives d sigma = Re(u^* dB v) with dB = dz I - dA, hence
//   d sigma / d Re z + i d sigma / d Im z = conj(u^* v),
//   d sigma / d Re A_ij + i d sigma / d Im A_ij = -u_i conj(v_j).
// sigma is the quantity of paper Sec. 2.1; these derivatives drive the Newton
// refinement of eps-contours (the level sets of paper Sec. 2, Definition
// "Pseudospectrum").
//
// Per point (one lane, as in k_sigma_min): banded LU, Lanczos on (B B^*)^{-1} to
// convergence; then
//   1. s = eigenvector of the Lanczos tridiagonal T_k for its top eigenvalue, by
//      inverse iteration on x I - T_k (x just above theta: positive definite, so
//      the tridiagonal LDL^T needs no pivoting);
//   2. a second pass replays the identical Lanczos recurrence (bit for bit) and
//      accumulates the Ritz vector y = sum_j s_j q_j = sum_j (s_j / beta_{j-1}) v_j;
//   3. u = y / |y| (the left singular vector: (B B^*)^{-1} has B's left singular
//      vectors as eigenvectors), v = B^{-1} u / |B^{-1} u|;
//   4. grad_z = sum_i u_i conj(v_i); for every band entry (i, i+d) the weighted
//      contribution -w u_i conj(v_{i+d}) is summed over the warp's 32 points with
//      shuffles and added to grad_bands with one atomic per entry and warp;
//   5. optionally u and v themselves are written out, so that band gradients for
//      other weights later need only the contraction k_band_grad_pairs.
#pragma once
#include "psa_kernel.cuh"

namespace psa {
namespace dev {

template <int KL, int KU>
__global__ void __launch_bounds__(kThreads, 2) k_sigma_min_grad(const KParams p)
{
    using SH = Shape<KL, KU>;
    constexpr int KW = SH::KW;
    constexpr int FX = SH::FX, FY = SH::FY;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n = p.n;
    const int RB = p.row_bytes;
    char *const wbase = p.wdata + warp * p.warp_bytes;
    char *const rows = wbase + lane * 16;
    uint8_t *const pivs = reinterpret_cast<uint8_t *>(wbase) + p.piv_offset + lane;
    double *const Ta = reinterpret_cast<double *>(wbase + (int64_t)p.trow * RB) + lane;
    const Mat M = single_mat(p);
    double *const Tb = Ta + (int64_t)p.k_max * 32;
    double *const Tc = Tb + (int64_t)p.k_max * 32;  // eigenvector s, then the coefficients s_j / beta_{j-1}
    double *const Td = Tc + (int64_t)p.k_max * 32;  // LDL^T pivots of x I - T_k
    constexpr int64_t TS = 32;
    const bool bad_input = p.flags[0] != 0;
    __shared__ double2 Aw_all[kThreads / 32][KW + 1][32];
    double2 (*const Aw)[32] = Aw_all[threadIdx.x >> 5];

#define FLD(j, f) (*reinterpret_cast<double2 *>(rows + (j) * RB + (f) * 512))
#define PIVOF(j) (pivs[(j) * RB])

    for (;;) {
        int grp = 0;
        if (lane == 0) grp = atomicAdd(p.counter, 1);
        grp = __shfl_sync(0xffffffffu, grp, 0);
        if ((int64_t)grp * 32 >= p.npts) break;
        const int64_t pt = (int64_t)grp * 32 + lane;
        const bool have = pt < p.npts;
        double zr = 0.0, zi = 0.0;
        if (have) {
            const double2 z = p.zpts[pt];
            zr = z.x;
            zi = z.y;
        }
        const bool singular = band_lu<KL, KU>(p, M, rows, pivs, Aw, lane, zr, zi, bad_input);
        // Lanes leave the Lanczos loops at their own step counts. Without a barrier the
        // lanes that are done would run ahead into the next phase while the others still
        // iterate, and the warp would issue both phases' FP64 instructions one after the
        // other (each costs the whole warp's FP64 slot whatever the active lanes): the
        // warp is brought back together after the first pass and around the replay.
        const unsigned live = __ballot_sync(0xffffffffu, have && !singular && !bad_input);

        double sigma = 0.0;
        int status = bad_input ? 3 : 1;
        int ksteps = 0;
        bool ok = false;
        double2 gz = make_double2(0.0, 0.0);
        double wgt = 0.0, inv_nx = 0.0;
        if (have && !singular && !bad_input) {
            LzState st;
            double theta = 0.0;
            status = lanczos_sigma<KL, KU>(p, M, rows, pivs, Ta, Tb, st, sigma, ksteps, theta);
            __syncwarp(live);
            ok = (status == 0 || status == 2) && sigma > 0.0 && ksteps >= 1;
            const unsigned okm = __ballot_sync(live, ok);
            if (ok) {
                // ---- 1. s = top eigenvector of T_k: two steps of inverse iteration on M = x I - T_k
                const int k = ksteps;
                const double x = theta + theta * 0x1.0p-44;
                double m = x - Ta[0];
                Td[0] = m;
                for (int i = 1; i < k; ++i) {
                    m = (x - Ta[(int64_t)i * TS]) - Tb[(int64_t)(i - 1) * TS] / m;
                    if (!(m > 0.0)) m = x * 0x1.0p-52;
                    Td[(int64_t)i * TS] = m;
                }
                for (int i = 0; i < k; ++i) Tc[(int64_t)i * TS] = 1.0;
                for (int it = 0; it < 2; ++it) {
                    // forward: y_i = b_i + (beta_{i-1} / m_{i-1}) y_{i-1}
                    double yprev = Tc[0];
                    for (int i = 1; i < k; ++i) {
                        const double bi = sqrt(Tb[(int64_t)(i - 1) * TS]);
                        yprev = fma(bi / Td[(int64_t)(i - 1) * TS], yprev, Tc[(int64_t)i * TS]);
                        Tc[(int64_t)i * TS] = yprev;
                    }
                    // back: s_i = y_i / m_i + (beta_i / m_i) s_{i+1}
                    double snext = Tc[(int64_t)(k - 1) * TS] / Td[(int64_t)(k - 1) * TS];
                    Tc[(int64_t)(k - 1) * TS] = snext;
                    double nrm = snext * snext;
                    for (int i = k - 2; i >= 0; --i) {
                        const double bi = sqrt(Tb[(int64_t)i * TS]);
                        snext = (Tc[(int64_t)i * TS] + bi * snext) / Td[(int64_t)i * TS];
                        Tc[(int64_t)i * TS] = snext;
                        nrm = fma(snext, snext, nrm);
                    }
                    const double inv = 1.0 / sqrt(nrm);
                    for (int i = 0; i < k; ++i) Tc[(int64_t)i * TS] *= inv;
                }
                // ---- coefficients of the stored vectors: v_1 = q_1, v_j = beta_{j-1} q_j
                for (int i = 1; i < k; ++i) Tc[(int64_t)i * TS] /= sqrt(Tb[(int64_t)(i - 1) * TS]);

                // ---- 2. second pass: y = sum_j c_j v_j into FY (same recurrence, same bits)
                __syncwarp(okm);
                LzState st2;
                for (int j = 1; j <= k; ++j) {
                    double a2;
                    (void)lanczos_step<KL, KU, true>(p, M, rows, pivs, Ta, Tb, j, st2, a2, Tc[(int64_t)(j - 1) * TS], j == k);
                }
                __syncwarp(okm);

                // ---- 3. u = y / |y| (kept in FY), x = B^{-1} (2^-e1 u) in FX, v = x / |x|
                double ny = 0.0;
                for (int i = 0; i < n; ++i) {
                    const double2 y = FLD(i, FY);
                    ny = fma(y.x, y.x, fma(y.y, y.y, ny));
                }
                const double invy = 1.0 / sqrt(ny);
                const double su = invy * pow2i(clampi(-st.e1, -1022, 1023));
                {
                    double2 X[KL + 1];
#pragma unroll
                    for (int r = 0; r <= KL; ++r) X[r] = make_double2(0.0, 0.0);
                    auto take = [&](int ii) -> double2 {
                        const double2 y = FLD(ii, FY);
                        FLD(ii, FY) = make_double2(y.x * invy, y.y * invy);
                        return make_double2(y.x * su, y.y * su);
                    };
#pragma unroll
                    for (int r = 0; r < KL; ++r)
                        if (r < n) X[r] = take(r);
                    for (int j = 0; j < n; ++j) {
                        X[KL] = (j + KL < n) ? take(j + KL) : make_double2(0.0, 0.0);
                        if (KL > 0) {
                            const int pj = PIVOF(j);
#pragma unroll
                            for (int r = 1; r <= KL; ++r) {
                                const bool s = (pj == r);
                                const double2 a = X[0], b = X[r];
                                X[0] = s ? b : a;
                                X[r] = s ? a : b;
                            }
#pragma unroll
                            for (int r = 1; r <= KL; ++r) X[r] = c_sub_mul(X[r], FLD(j, KW + r), X[0]);
                        }
                        FLD(j, FX) = X[0];
#pragma unroll
                        for (int r = 0; r < KL; ++r) X[r] = X[r + 1];
                    }
                }
                double nx = 0.0;
                {
                    double2 Y[KW + 1];
#pragma unroll
                    for (int c = 0; c <= KW; ++c) Y[c] = make_double2(0.0, 0.0);
                    for (int j = n - 1; j >= 0; --j) {
                        double2 acc = FLD(j, FX);
#pragma unroll
                        for (int c = 1; c <= KW; ++c) acc = c_sub_mul(acc, FLD(j, c), Y[c]);
                        const double2 xv = c_mul(acc, FLD(j, 0));
                        nx = fma(xv.x, xv.x, fma(xv.y, xv.y, nx));
                        FLD(j, FX) = xv;
#pragma unroll
                        for (int c = KW; c >= 2; --c) Y[c] = Y[c - 1];
                        if (KW >= 1) Y[1] = xv;
                    }
                }
                inv_nx = 1.0 / sqrt(nx);
                // ---- 4. grad_z = sum_i u_i conj(v_i)
                for (int i = 0; i < n; ++i) {
                    const double2 u = FLD(i, FY);
                    const double2 xv = FLD(i, FX);
                    gz.x = fma(u.x, xv.x, fma(u.y, xv.y, gz.x));
                    gz.y = fma(u.y, xv.x, fma(-u.x, xv.y, gz.y));
                }
                gz.x *= inv_nx;
                gz.y *= inv_nx;
                wgt = p.gweight ? p.gweight[pt] : 0.0;
            }
        }
        __syncwarp();
        // ---- the singular pair itself (u, v = x / |x|), element-major so that a warp's
        //      32 points write 32 consecutive values of each row
        if (p.u_out && have) {
            for (int i = 0; i < n; ++i) {
                const double2 u = ok ? FLD(i, FY) : make_double2(0.0, 0.0);
                const double2 xv = ok ? FLD(i, FX) : make_double2(0.0, 0.0);
                p.u_out[(int64_t)i * p.npts + pt] = u;
                p.v_out[(int64_t)i * p.npts + pt] = make_double2(xv.x * inv_nx, xv.y * inv_nx);
            }
        }

        // ---- band gradient: all 32 lanes take part in the shuffles
        if (p.grad_bands) {
            const double cw = ok ? -wgt * inv_nx : 0.0;  // -w / |x| (v = x / |x|)
            for (int i = 0; i < n; ++i) {
                const double2 u = ok ? FLD(i, FY) : make_double2(0.0, 0.0);
#pragma unroll
                for (int dd = 0; dd <= KW; ++dd) {
                    const int d = dd - KL;  // band entry (i, i + d)
                    const int j = i + d;
                    if (j < 0 || j >= n) continue;  // uniform across the warp
                    const double2 xv = ok ? FLD(j, FX) : make_double2(0.0, 0.0);
                    // -w u_i conj(v_j)
                    double gx = cw * fma(u.x, xv.x, u.y * xv.y);
                    double gy = cw * fma(u.y, xv.x, -(u.x * xv.y));
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) {
                        gx += __shfl_xor_sync(0xffffffffu, gx, off);
                        gy += __shfl_xor_sync(0xffffffffu, gy, off);
                    }
                    if (lane == (dd & 31)) {
                        double2 *const tgt = p.grad_bands + (int64_t)dd * n + i;
                        atomicAdd(&tgt->x, gx);
                        atomicAdd(&tgt->y, gy);
                    }
                }
            }
        }

        if (have) {
            p.sigma[pt] = sigma;
            if (p.grad_z) p.grad_z[pt] = ok ? gz : make_double2(0.0, 0.0);
            if (p.status) p.status[pt] = (int8_t)status;
            if (p.steps) p.steps[pt] = ksteps;
        }
    }
#undef FLD
#undef PIVOF
}

template <int KL, int KU>
cudaError_t launch_sigma_min_grad(const KParams &p, cudaStream_t stream)
{
    const int threads = (p.P % kThreads == 0) ? kThreads : 32;
    k_sigma_min_grad<KL, KU><<<(unsigned)(p.P / threads), threads, 0, stream>>>(p);
    return cudaGetLastError();
}

template <int KL, int KU>
cudaError_t grad_blocks_per_sm(int *nb)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_sigma_min_grad<KL, KU>, kThreads, 0);
}

}  // namespace dev

template <int KL>
KernelOps grad_ops_for_ku(int ku)
{
    switch (ku) {
#define PSA_KU_CASE(K) case K: return KernelOps{&dev::launch_sigma_min_grad<KL, K>, &dev::grad_blocks_per_sm<KL, K>};
    PSA_KU_CASE(0) PSA_KU_CASE(1) PSA_KU_CASE(2) PSA_KU_CASE(3) PSA_KU_CASE(4)
    PSA_KU_CASE(5) PSA_KU_CASE(6) PSA_KU_CASE(7) PSA_KU_CASE(8)
#undef PSA_KU_CASE
    default: return KernelOps{nullptr, nullptr};
    }
}

}  // namespace psa
