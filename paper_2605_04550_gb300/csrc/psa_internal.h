// psa_internal.h -- types shared by the translation units of libpsa (not public).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace psa {

constexpr int kMaxEps = 32;
constexpr int kThreads = 128;        // threads per block of the sigma_min kernel
constexpr int kMaxKL = 4;            // compile-time band shapes: kl in [0, 4]
constexpr int kMaxKU = 8;            //                           ku in [0, 8]

// Everything one launch of the sigma_min kernel needs (passed by value).
struct KParams {
    // matrix: bands[(d + kl) * n + i] = A[i][i + d]
    const double2 *bands;
    int n, kl, ku;
    // grid
    double re_min, im_min, hx, hy;
    int nx, ny;
    // points: idx == nullptr -> flat index = point number; else idx[point]
    const int32_t *idx;
    int64_t npts;
    // epsilon levels
    double eps[kMaxEps];
    int n_eps;
    // Lanczos controls
    int k_min, k_max;
    double tol;
    // outputs (flat grid index)
    double *sigma;
    uint32_t *mask;
    int8_t *status;
    int32_t *steps;
    // workspace: per slot t in [0, P), every array is [row][P] (row-major in row,
    // slot fastest) so that a warp touches 32 consecutive slots per access
    const int *flags;   // flags[0] != 0: a band entry of A is not finite
    const double2 *q1;  // start vector, n values (shared by all slots)
    double2 *F;         // factor rows: [n][S][P], S = 2kl + ku + 1
    uint8_t *piv;       // pivot offsets: [n][P]
    double2 *Va, *Vb, *Vx;  // Lanczos vectors: [n][P] each
    double *Ta, *Tb;    // alpha_k, beta_k^2: [k_max][P] each
    int64_t P;
};

using launch_fn = cudaError_t (*)(const KParams &, cudaStream_t);

// One launcher per compiled (kl, ku); defined in psa_inst_kl*.cu.
launch_fn launcher_kl0(int ku);
launch_fn launcher_kl1(int ku);
launch_fn launcher_kl2(int ku);
launch_fn launcher_kl3(int ku);
launch_fn launcher_kl4(int ku);

}  // namespace psa
