// psa_internal.h -- types shared by the translation units of libpsa (not public).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace psa {

constexpr int kMaxEps = 32;
constexpr int kThreads = 128;        // threads per block of the sigma_min kernel
// Resident blocks per SM of one launch: 2 blocks of 4 warps = 2 warps per scheduler.
// Two warps keep a scheduler's FP64 unit about 94 % busy; a third adds ~2 % in the
// steady state but makes every warp run at a third of the unit, so the longest groups
// (hundreds of Lanczos steps, started first) end up to 1.2 s after the rest of the
// launch on the n = 2000 grid (4.27 s per grid with 3 warps, 3.63 s with 2).
constexpr int kBlocksPerSm = 2;
constexpr int kMaxKL = 4;            // compile-time band shapes: kl in [0, 4]
constexpr int kMaxKU = 8;            //                           ku in [0, 8]
constexpr int kBuckets = 4096;       // cost buckets of the work order (matrix order x sigma)
constexpr int kMaxStreams = 8;       // batches: the caller's stream and up to 7 auxiliary streams

// One matrix of a batch, as the device plan lists it (psa_batch_plan): matrices of
// one band shape are consecutive, gstart is the first group of the matrix within
// its class, q1_off the offset (in complex values) of its start vector in the
// workspace, out_off the first index of its outputs.
struct PlanMat {
    const double2 *bands;
    int32_t n, nx, ny, pad;
    double re_min, im_min, hx, hy;
    int64_t out_off, gstart, q1_off;
    int64_t estart;  // first estimate chunk (32 anchors of this matrix) within its class
};

// A band-shape class of a batch plan: matrices first .. first+count-1 of the plan.
struct PlanClass {
    int32_t kl, ku, n_max, first, count, pad;
    int64_t ngroups, nchunks;
};

// Plan memory (host and device copies are identical): header, kMaxClasses classes,
// then one PlanMat per matrix (class by class).
constexpr int kMaxClasses = (kMaxKL + 1) * (kMaxKU + 1);
constexpr int32_t kPlanMagic = 0x50534142;
struct PlanHeader {
    int32_t magic, nmat, nclass, max_n;
    int64_t q1_total;      // complex values of all start vectors
    int64_t max_ngroups;   // groups of the largest class
};
constexpr size_t kPlanClassOff = 256;
constexpr size_t kPlanMatOff = kPlanClassOff + ((kMaxClasses * sizeof(PlanClass) + 255) / 256) * 256;

// Everything one launch of the sigma_min kernel needs (passed by value).
struct KParams {
    // matrix: bands[(d + kl) * n + i] = A[i][i + d]
    const double2 *bands;
    int n, kl, ku;
    // grid
    double re_min, im_min, hx, hy;
    int nx, ny;
    // batch: nmats > 0 -> groups are tiles of the matrices pmats[0 .. nmats) (one band
    // shape), whose start vectors sit at q1 + pmats[m].q1_off; trow = rows of the
    // largest matrix (the tridiagonal arrays of a warp block follow them)
    const PlanMat *pmats;
    int nmats;
    int trow;
    const int *mflags;  // batch: mflags[m] != 0 when matrix m has a non-finite band entry
    // points: idx == nullptr -> flat index = point number; else idx[point]
    const int32_t *idx;
    int64_t npts;
    int64_t ngroups;  // groups of 32 points: 8 x 4 grid tiles (full grid) or list chunks
    int64_t nchunks;  // estimate pass: chunks of 32 anchors
    // work order: estimate != 0 runs only each group's anchor point for k_max steps
    // and files the group under a cost bucket (matrix order, then sigma relative to
    // the grid's extent: sched_bucket, sched_hist);
    // otherwise warps take groups order[0], order[1], ... (or 0, 1, ... if order is NULL)
    int estimate;
    const int *order;
    int *sched_bucket;
    int *sched_hist;
    // epsilon levels
    double eps[kMaxEps];
    int n_eps;
    // Lanczos controls
    int k_min, k_max;
    double tol;
    // gradient kernel: explicit points z (zpts), upstream weights, outputs by point
    const double2 *zpts;
    const double *gweight;
    double2 *grad_z;
    double2 *grad_bands;
    double2 *u_out, *v_out;  // gradient kernel: the singular pair, u_out[i * npts + pt] (or null)
    // outputs (flat grid index; point index for the gradient kernel)
    double *sigma;
    uint32_t *mask;
    int8_t *status;
    int32_t *steps;
    // workspace
    const int *flags;   // flags[0] != 0: a band entry of A is not finite
    int *counter;       // next group of 32 points (zeroed before the launch)
    const double2 *q1;  // start vector, n values (shared by all warps)
    char *wdata;        // per-warp blocks of warp_bytes, row records of row_bytes
    int64_t warp_bytes;
    int row_bytes;
    int piv_offset;     // byte offset of the pivot bytes inside a row record
    int64_t P;          // threads launched (a multiple of kThreads)
};

struct KernelOps {
    cudaError_t (*launch)(const KParams &, cudaStream_t);
    cudaError_t (*blocks_per_sm)(int *);  // resident blocks of kThreads per SM
};

}  // namespace psa
#include "psa.h"
namespace psa {
// Argument checks of psa_sigma_min other than the workspace (PSA_OK or the code that
// psa_sigma_min would return); psa_abi.cu.
int check_sigma_min_args(const psa_band *A, const psa_grid *g, const double *eps, int32_t n_eps,
                         const int32_t *idx, int64_t n_idx, const double *sigma, const psa_lanczos_opts *opts);

// One entry per compiled (kl, ku); defined in psa_inst_kl*.cu (sigma_min) and
// psa_grad_kl*.cu (sigma_min with gradients).
KernelOps kernel_ops_kl0(int ku);
KernelOps kernel_ops_kl1(int ku);
KernelOps kernel_ops_kl2(int ku);
KernelOps kernel_ops_kl3(int ku);
KernelOps kernel_ops_kl4(int ku);
KernelOps grad_ops_kl0(int ku);
KernelOps grad_ops_kl1(int ku);
KernelOps grad_ops_kl2(int ku);
KernelOps grad_ops_kl3(int ku);
KernelOps grad_ops_kl4(int ku);

}  // namespace psa
