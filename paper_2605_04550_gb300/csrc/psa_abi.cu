// psa_abi.cu -- the C ABI of libpsa: argument checks, workspace layout,
// set-up kernels and dispatch of the sigma_min kernel by band shape.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

#include "psa.h"
#include "psa_internal.h"
#include "psa_kernel.cuh"

namespace psa {
namespace {

constexpr size_t kAlign = 256;
constexpr int kEstimateSteps = 4;  // Lanczos steps of the work-order estimate
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace: [flags: 256 B][schedule][q1: n complex][per-warp blocks]. flags[0] marks
// a non-finite band entry, flags[1] and flags[2] are the group counters of the main
// and estimate passes. The schedule (optional) holds the bucket histogram and
// cursors (kBuckets ints each), then one bucket and one order slot per group. A warp
// block holds n row records of row_bytes, then alpha_k and beta_k^2 for k_max steps
// (see the kernel's header comment).
struct Layout {
    size_t flags, sched, q1, wdata, total;
    int64_t warp_bytes;
    int row_bytes;
};

// Row record: S = 2kl+ku+1 factor fields and nvec Lanczos vector fields of 512 bytes,
// then 32 pivot bytes (padded to 128).
int row_bytes_of(int kl, int ku, int nvec = 3) { return (2 * kl + ku + 1 + nvec) * 512 + 128; }

size_t sched_bytes(int64_t ngroups)
{
    return ngroups > 0 ? align_up(sizeof(int) * (2 * (size_t)kBuckets + 2 * (size_t)ngroups)) : 0;
}

Layout layout(int64_t n, int kl, int ku, int kmax, int64_t nwarps, int64_t ngroups, int nvec = 3, int ntri = 2)
{
    Layout L{};
    L.row_bytes = row_bytes_of(kl, ku, nvec);
    L.warp_bytes = (int64_t)align_up((size_t)n * L.row_bytes + (size_t)ntri * (size_t)kmax * 32 * sizeof(double));
    size_t off = 0;
    L.flags = off; off += kAlign;
    L.sched = off; off += sched_bytes(ngroups);
    L.q1 = off;    off += align_up(sizeof(double2) * (size_t)n);
    L.wdata = off; off += (size_t)nwarps * L.warp_bytes;
    L.total = off;
    return L;
}

// Upper bound on the groups of a call with `npoints` points: list chunks of 32, or
// 8 x 4 tiles of an nx x ny grid (at most npoints / 8 + 2 of them).
int64_t max_groups(int64_t npoints) { return npoints > 0 ? npoints / 8 + 2 : 0; }

bool band_ok(const psa_band *A)
{
    return A && A->n >= 1 && A->kl >= 0 && A->ku >= 0 && A->kl <= A->n - 1 && A->ku <= A->n - 1;
}

// Row offsets inside a warp block are 32-bit.
bool fits_row_offsets(const psa_band *A)
{
    return (int64_t)A->n * row_bytes_of(A->kl, A->ku) < 2147483647LL;
}

bool opts_ok(const psa_lanczos_opts &o)
{
    return o.k_max >= 1 && o.k_max <= 65535 && o.k_min >= 0 && o.k_min <= o.k_max && std::isfinite(o.tol) &&
           o.tol >= 0.0;
}

int64_t round_down(int64_t v, int64_t m) { return v / m * m; }

// ----------------------------------------------------------- set-up kernels
__device__ __forceinline__ double unit_interval(unsigned long long v)
{
    return __ull2double_rn(v >> 11) * 0x1.0p-52 - 1.0;
}

// q1 = h / |h|, h_i = u(2i) + i u(2i+1), by one block of 256 threads with a
// fixed-order reduction (the same bits for a matrix alone and in a batch).
__device__ __forceinline__ void start_vector_block(double2 *q1, int n, unsigned long long seed)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const double re = unit_interval(dev::splitmix64(seed, 2ULL * (unsigned long long)i));
        const double im = unit_interval(dev::splitmix64(seed, 2ULL * (unsigned long long)i + 1ULL));
        q1[i] = make_double2(re, im);
        s = fma(re, re, fma(im, im, s));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double inv = 1.0 / sqrt(red[0]);
    for (int i = threadIdx.x; i < n; i += 256) {
        const double2 h = q1[i];
        q1[i] = make_double2(h.x * inv, h.y * inv);
    }
}

__global__ void __launch_bounds__(256) k_start_vector(double2 *q1, int n, unsigned long long seed)
{
    start_vector_block(q1, n, seed);
}

// flags[0] |= 1 when a band entry A[i][i+d] (0 <= i+d < n) is not finite.
__global__ void k_check_finite(const double2 *bands, int n, int kl, int ku, int *flags)
{
    const int64_t total = (int64_t)(kl + ku + 1) * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int dk = (int)(e / n);
        const int i = (int)(e - (int64_t)dk * n);
        const int col = i + dk - kl;
        if (col < 0 || col >= n) continue;
        const double2 a = bands[e];
        if (!isfinite(a.x) || !isfinite(a.y)) atomicOr(flags, 1);
    }
}

// cursor[b] = number of groups in buckets above b (descending order of buckets):
// one block of 1024 threads, thread t owns buckets 4t .. 4t+3; an inclusive scan of
// the per-thread sums from the top (Hillis-Steele in shared memory) gives each
// thread the count above its buckets.
constexpr int kScanThreads = 1024;
static_assert(kBuckets == 4 * kScanThreads, "k_sched_scan: 4 buckets per thread");
__global__ void __launch_bounds__(kScanThreads) k_sched_scan(const int *hist, int *cursor)
{
    __shared__ int s[2][kScanThreads];
    const int t = threadIdx.x;
    const int4 h = reinterpret_cast<const int4 *>(hist)[t];
    // thread index r = 1023 - t so that the scan runs from the highest buckets down
    const int r = kScanThreads - 1 - t;
    s[0][r] = h.x + h.y + h.z + h.w;
    __syncthreads();
    int cur = 0;
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const int v = s[cur][r] + (r >= off ? s[cur][r - off] : 0);
        s[cur ^ 1][r] = v;
        cur ^= 1;
        __syncthreads();
    }
    const int above = s[cur][r] - (h.x + h.y + h.z + h.w);  // buckets > 4t + 3
    int4 c;
    c.w = above;
    c.z = c.w + h.w;
    c.y = c.z + h.z;
    c.x = c.y + h.y;
    reinterpret_cast<int4 *>(cursor)[t] = c;
}

// order[slot] = group, groups of higher buckets first (order within a bucket is
// immaterial: it changes which warp takes a group, never a point's result).
__global__ void k_sched_scatter(const int *bucket, int *cursor, int *order, int64_t ngroups)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < ngroups; a += (int64_t)gridDim.x * blockDim.x) {
        const int b = bucket[a] & (kBuckets - 1);
        order[atomicAdd(&cursor[b], 1)] = (int)a;
    }
}

// Restricted mode: every point starts as "not evaluated" (paper Sec. 4: points
// outside the predicted region are classified non-sensitive).
__global__ void k_fill_not_evaluated(double *sigma, uint32_t *mask, int8_t *status, int32_t *steps, int64_t N)
{
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        sigma[i] = qnan;
        if (mask) mask[i] = 0u;
        if (status) status[i] = (int8_t)PSA_PT_NOT_EVALUATED;
        if (steps) steps[i] = 0;
    }
}

// Batch start vectors, one block per matrix of the plan (as k_start_vector).
__global__ void __launch_bounds__(256) k_batch_start_vectors(const PlanMat *mats, double2 *q1,
                                                             unsigned long long seed)
{
    const PlanMat &e = mats[blockIdx.x];
    start_vector_block(q1 + e.q1_off, e.n, seed);
}

// Batch input check of one class (band shape kl, ku): blockIdx.y = matrix within the
// class, blocks in x stride over its band entries.
__global__ void k_batch_check_finite(const PlanMat *mats, int kl, int ku, int *mflags)
{
    const PlanMat &e = mats[blockIdx.y];
    const int n = e.n;
    const int64_t total = (int64_t)(kl + ku + 1) * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int dk = (int)(q / n);
        const int i = (int)(q - (int64_t)dk * n);
        const int col = i + dk - kl;
        if (col < 0 || col >= n) continue;
        const double2 a = e.bands[q];
        if (!isfinite(a.x) || !isfinite(a.y)) atomicOr(&mflags[blockIdx.y], 1);
    }
}

__device__ double g_probe_sink;

// Independent DFMA chains: 8 per thread.
__global__ void k_probe_dfma(int iters, double m, double c)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 1.2345678e-300) g_probe_sink = s;  // keeps the chains live
}

KernelOps pick_ops(int kl, int ku)
{
    switch (kl) {
    case 0: return kernel_ops_kl0(ku);
    case 1: return kernel_ops_kl1(ku);
    case 2: return kernel_ops_kl2(ku);
    case 3: return kernel_ops_kl3(ku);
    case 4: return kernel_ops_kl4(ku);
    default: return KernelOps{nullptr, nullptr};
    }
}

KernelOps pick_grad_ops(int kl, int ku)
{
    switch (kl) {
    case 0: return grad_ops_kl0(ku);
    case 1: return grad_ops_kl1(ku);
    case 2: return grad_ops_kl2(ku);
    case 3: return grad_ops_kl3(ku);
    case 4: return grad_ops_kl4(ku);
    default: return KernelOps{nullptr, nullptr};
    }
}

// Threads that fill the device once with the kernel for (kl, ku): the resident
// blocks per SM that the occupancy allows, at most kBlocksPerSm.
int full_threads(const KernelOps &ops, int64_t *out)
{
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSA_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PSA_ECUDA;
    if (ops.blocks_per_sm(&nb) != cudaSuccess || nb < 1) return PSA_ECUDA;
    if (nb > kBlocksPerSm) nb = kBlocksPerSm;
    *out = (int64_t)sms * nb * kThreads;
    return PSA_OK;
}

}  // namespace
}  // namespace psa

namespace psa {
// The argument checks of psa_sigma_min (everything but the workspace), shared with
// psa_sigma_min_static so that both report the same codes.
int check_sigma_min_args(const psa_band *A, const psa_grid *g, const double *eps, int32_t n_eps,
                         const int32_t *idx, int64_t n_idx, const double *sigma, const psa_lanczos_opts *opts)
{
    if (!band_ok(A) || !A->bands || !g || !sigma) return PSA_EINVAL;
    if (!(std::isfinite(g->re_min) && std::isfinite(g->re_max) && std::isfinite(g->im_min) &&
          std::isfinite(g->im_max)) ||
        g->re_min > g->re_max || g->im_min > g->im_max || g->nx < 1 || g->ny < 1)
        return PSA_EINVAL;
    if ((int64_t)g->nx * g->ny > 2147483647LL) return PSA_EINVAL;
    if (n_eps < 0 || n_eps > kMaxEps || (n_eps > 0 && !eps)) return PSA_EINVAL;
    for (int l = 0; l < n_eps; ++l)
        if (!std::isfinite(eps[l]) || !(eps[l] > 0.0)) return PSA_EINVAL;
    if (n_idx < 0 || (n_idx > 0 && !idx)) return PSA_EINVAL;
    if (!opts_ok(opts ? *opts : psa_default_opts())) return PSA_EINVAL;
    if (A->kl > kMaxKL || A->ku > kMaxKU || !fits_row_offsets(A)) return PSA_EUNSUPPORTED;
    if (!pick_ops(A->kl, A->ku).launch) return PSA_EUNSUPPORTED;
    return PSA_OK;
}
}  // namespace psa

using namespace psa;

extern "C" {

int psa_version(void) { return 100; }

const char *psa_strerror(int code)
{
    switch (code) {
    case PSA_OK: return "ok";
    case PSA_EINVAL: return "invalid argument";
    case PSA_EWORKSPACE: return "workspace too small";
    case PSA_ECUDA: return "CUDA error";
    case PSA_EUNSUPPORTED: return "unsupported band shape (kl <= 4, ku <= 8)";
    case PSA_ESTATIC: return "problem too large for the static scratch of psa_sigma_min_static";
    default: return "unknown error";
    }
}

psa_lanczos_opts psa_default_opts(void)
{
    psa_lanczos_opts o;
    o.k_min = 2;
    o.k_max = 1000;
    o.tol = 1e-13;
    o.seed = 0;
    return o;
}

int psa_workspace_bytes(const psa_band *A, const psa_lanczos_opts *opts, int64_t points_in_flight, int64_t npoints,
                        size_t *bytes)
{
    if (!band_ok(A) || points_in_flight < 1 || npoints < 0 || !bytes) return PSA_EINVAL;
    const psa_lanczos_opts o = opts ? *opts : psa_default_opts();
    if (!opts_ok(o)) return PSA_EINVAL;
    const int64_t nwarps = (points_in_flight + 31) / 32;
    *bytes = layout(A->n, A->kl, A->ku, o.k_max, nwarps, max_groups(npoints)).total;
    return PSA_OK;
}

int psa_default_points_in_flight(const psa_band *A, int64_t npoints, int64_t *out)
{
    if (!band_ok(A) || npoints < 1 || !out) return PSA_EINVAL;
    if (A->kl > kMaxKL || A->ku > kMaxKU) return PSA_EUNSUPPORTED;
    const KernelOps ops = pick_ops(A->kl, A->ku);
    if (!ops.launch) return PSA_EUNSUPPORTED;
    int64_t full = 0;
    const int rc = full_threads(ops, &full);
    if (rc != PSA_OK) return rc;
    const int64_t need = (npoints + 31) / 32 * 32;
    *out = need < full ? need : full;
    return PSA_OK;
}

int psa_sigma_min(const psa_band *A, const psa_grid *g, const double *eps, int32_t n_eps, const int32_t *idx,
                  int64_t n_idx, double *sigma, uint32_t *mask, int8_t *status, int32_t *steps,
                  const psa_lanczos_opts *opts, void *workspace, size_t ws_bytes, void *stream_ptr)
{
    const int arc = check_sigma_min_args(A, g, eps, n_eps, idx, n_idx, sigma, opts);
    if (arc != PSA_OK) return arc;
    const int64_t ngrid = (int64_t)g->nx * g->ny;
    const psa_lanczos_opts o = opts ? *opts : psa_default_opts();
    const KernelOps ops = pick_ops(A->kl, A->ku);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return PSA_EWORKSPACE;

    const int64_t npts = idx ? n_idx : ngrid;
    const int64_t n = A->n;
    // points in flight: whole warps, as many as the workspace holds, at most one
    // full occupancy of the device and no more than the points to evaluate
    const int64_t ngroups = idx ? (npts + 31) / 32 : (int64_t)((g->nx + 7) / 8) * ((g->ny + 3) / 4);
    const Layout L1 = layout(n, A->kl, A->ku, o.k_max, 1, 0);
    if (L1.total > ws_bytes) return PSA_EWORKSPACE;
    // the longest-first work order needs the schedule arrays; without room for them
    // (a workspace sized for no points) warps take the groups in grid order
    bool ordered = layout(n, A->kl, A->ku, o.k_max, 1, ngroups).total <= ws_bytes && ngroups > 1;
    const size_t sched = ordered ? sched_bytes(ngroups) : 0;
    int64_t nwarps = (int64_t)((ws_bytes - sched - (L1.total - (size_t)L1.warp_bytes)) / (size_t)L1.warp_bytes);
    int64_t full = 0;
    const int frc = full_threads(ops, &full);
    if (frc != PSA_OK) return frc;
    if (nwarps > full / 32) nwarps = full / 32;
    if (nwarps > ngroups) nwarps = ngroups < 1 ? 1 : ngroups;
    // the estimate pass pays off when warps take several groups each (a long tail)
    if (ordered && ngroups < 4 * nwarps) ordered = false;
    if (nwarps >= 4) nwarps = round_down(nwarps, 4);
    const Layout L = layout(n, A->kl, A->ku, o.k_max, nwarps, ordered ? ngroups : 0);
    const int64_t P = nwarps * 32;

    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    char *ws = static_cast<char *>(workspace);

    KParams p{};
    p.bands = reinterpret_cast<const double2 *>(A->bands);
    p.n = A->n;
    p.kl = A->kl;
    p.ku = A->ku;
    p.re_min = g->re_min;
    p.im_min = g->im_min;
    p.hx = g->nx > 1 ? (g->re_max - g->re_min) / (double)(g->nx - 1) : 0.0;
    p.hy = g->ny > 1 ? (g->im_max - g->im_min) / (double)(g->ny - 1) : 0.0;
    p.nx = g->nx;
    p.ny = g->ny;
    p.idx = idx;
    p.npts = npts;
    p.ngroups = ngroups;
    p.nchunks = (ngroups + 31) / 32;
    for (int l = 0; l < kMaxEps; ++l) p.eps[l] = l < n_eps ? eps[l] : 0.0;
    p.n_eps = n_eps;
    p.k_min = o.k_min;
    p.k_max = o.k_max;
    p.tol = o.tol;
    p.sigma = sigma;
    p.mask = n_eps > 0 ? mask : nullptr;
    p.status = status;
    p.steps = steps;
    p.flags = reinterpret_cast<const int *>(ws + L.flags);
    p.counter = reinterpret_cast<int *>(ws + L.flags) + 1;
    int *const hist = reinterpret_cast<int *>(ws + L.sched);
    int *const cursor = hist + kBuckets;
    int *const bucket = cursor + kBuckets;
    int *const order = bucket + ngroups;
    p.estimate = 0;
    p.order = ordered ? order : nullptr;
    p.sched_bucket = bucket;
    p.sched_hist = hist;
    p.q1 = reinterpret_cast<const double2 *>(ws + L.q1);
    p.wdata = ws + L.wdata;
    p.warp_bytes = L.warp_bytes;
    p.row_bytes = L.row_bytes;
    p.piv_offset = (2 * A->kl + A->ku + 1 + 3) * 512;
    p.trow = A->n;
    p.P = P;

    if (mask && n_eps == 0) {
        if (cudaMemsetAsync(mask, 0, sizeof(uint32_t) * (size_t)ngrid, stream) != cudaSuccess) return PSA_ECUDA;
    }
    if (idx) {
        const int64_t blocks = (ngrid + 255) / 256 < 4096 ? (ngrid + 255) / 256 : 4096;
        k_fill_not_evaluated<<<(unsigned)blocks, 256, 0, stream>>>(sigma, mask, status, steps, ngrid);
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    }
    k_start_vector<<<1, 256, 0, stream>>>(reinterpret_cast<double2 *>(ws + L.q1), A->n, o.seed);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    if (cudaMemsetAsync(ws + L.flags, 0, kAlign, stream) != cudaSuccess) return PSA_ECUDA;
    {
        const int64_t total = (int64_t)(A->kl + A->ku + 1) * A->n;
        const int64_t blocks = (total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024;
        k_check_finite<<<(unsigned)blocks, 256, 0, stream>>>(p.bands, A->n, A->kl, A->ku,
                                                              reinterpret_cast<int *>(ws + L.flags));
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    }
    if (npts == 0) return PSA_OK;
    if (ordered) {
        // estimate pass: each group's anchor point, LU + a few Lanczos steps, then the
        // groups sorted into decreasing buckets of log2(sigma estimate)
        if (cudaMemsetAsync(hist, 0, sizeof(int) * kBuckets, stream) != cudaSuccess) return PSA_ECUDA;
        KParams pe = p;
        pe.estimate = 1;
        pe.order = nullptr;
        pe.k_min = pe.k_max = o.k_max < kEstimateSteps ? o.k_max : kEstimateSteps;
        pe.tol = 0.0;
        pe.counter = reinterpret_cast<int *>(ws + L.flags) + 2;
        pe.sigma = nullptr;
        pe.mask = nullptr;
        pe.status = nullptr;
        pe.steps = nullptr;
        if (ops.launch(pe, stream) != cudaSuccess) return PSA_ECUDA;
        k_sched_scan<<<1, kScanThreads, 0, stream>>>(hist, cursor);
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
        const int64_t sb = (ngroups + 255) / 256 < 4096 ? (ngroups + 255) / 256 : 4096;
        k_sched_scatter<<<(unsigned)sb, 256, 0, stream>>>(bucket, cursor, order, ngroups);
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    }
    if (ops.launch(p, stream) != cudaSuccess) return PSA_ECUDA;
    return PSA_OK;
}

int psa_grad_workspace_bytes(const psa_band *A, const psa_lanczos_opts *opts, int64_t points_in_flight, size_t *bytes)
{
    if (!band_ok(A) || points_in_flight < 1 || !bytes) return PSA_EINVAL;
    const psa_lanczos_opts o = opts ? *opts : psa_default_opts();
    if (!opts_ok(o)) return PSA_EINVAL;
    const int64_t nwarps = (points_in_flight + 31) / 32;
    *bytes = layout(A->n, A->kl, A->ku, o.k_max, nwarps, 0, 4, 4).total;
    return PSA_OK;
}

}  // extern "C"

namespace psa {
namespace {

// grad_bands[(d + kl) * n + i] = -sum_p w[p] u[i][p] conj(v[i + d][p]): one warp per band
// entry, its lanes striding over the points (element-major u, v: coalesced reads),
// then a fixed-order shuffle sum (the same bits on every run).
__global__ void k_band_grad_pairs(int n, int kl, int ku, int64_t npts, const double2 *u, const double2 *v,
                                  const double *w, double2 *g)
{
    const int64_t nent = (int64_t)(kl + ku + 1) * n;
    const int lane = threadIdx.x & 31;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nent;
         e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int dk = (int)(e / n), i = (int)(e - (int64_t)dk * n);
        const int j = i + dk - kl;
        double gx = 0.0, gy = 0.0;
        if (j >= 0 && j < n) {
            const double2 *ui = u + (int64_t)i * npts, *vj = v + (int64_t)j * npts;
            for (int64_t q = lane; q < npts; q += 32) {
                const double2 a = ui[q], b = vj[q];
                const double c = -w[q];
                gx = fma(c, fma(a.x, b.x, a.y * b.y), gx);
                gy = fma(c, fma(a.y, b.x, -(a.x * b.y)), gy);
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, off);
            gy += __shfl_xor_sync(0xffffffffu, gy, off);
        }
        if (lane == 0) g[e] = make_double2(gx, gy);
    }
}

int sigma_min_grad_impl(const psa_band *A, const psa_c64 *z, int64_t n_pts, const double *weight, double *sigma,
                        psa_c64 *grad_z, psa_c64 *grad_bands, psa_c64 *u_out, psa_c64 *v_out, int8_t *status,
                        int32_t *steps, const psa_lanczos_opts *opts, void *workspace, size_t ws_bytes,
                        void *stream_ptr)
{
    if (!band_ok(A) || !A->bands || n_pts < 0 || (n_pts > 0 && (!z || !sigma))) return PSA_EINVAL;
    if (grad_bands && !weight) return PSA_EINVAL;
    const psa_lanczos_opts o = opts ? *opts : psa_default_opts();
    if (!opts_ok(o)) return PSA_EINVAL;
    if (A->kl > kMaxKL || A->ku > kMaxKU || (int64_t)A->n * row_bytes_of(A->kl, A->ku, 4) >= 2147483647LL)
        return PSA_EUNSUPPORTED;
    const KernelOps ops = pick_grad_ops(A->kl, A->ku);
    if (!ops.launch) return PSA_EUNSUPPORTED;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return PSA_EWORKSPACE;
    const int64_t n = A->n;
    const Layout L1 = layout(n, A->kl, A->ku, o.k_max, 1, 0, 4, 4);
    if (L1.total > ws_bytes) return PSA_EWORKSPACE;
    int64_t nwarps = (int64_t)((ws_bytes - (L1.total - (size_t)L1.warp_bytes)) / (size_t)L1.warp_bytes);
    int64_t full = 0;
    const int frc = full_threads(ops, &full);
    if (frc != PSA_OK) return frc;
    if (nwarps > full / 32) nwarps = full / 32;
    const int64_t ngroups = (n_pts + 31) / 32;
    if (nwarps > ngroups) nwarps = ngroups < 1 ? 1 : ngroups;
    if (nwarps >= 4) nwarps = round_down(nwarps, 4);
    const Layout L = layout(n, A->kl, A->ku, o.k_max, nwarps, 0, 4, 4);
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    char *ws = static_cast<char *>(workspace);

    KParams p{};
    p.bands = reinterpret_cast<const double2 *>(A->bands);
    p.n = A->n;
    p.kl = A->kl;
    p.ku = A->ku;
    p.nx = 1;
    p.ny = 1;
    p.npts = n_pts;
    p.ngroups = ngroups;
    p.nchunks = (ngroups + 31) / 32;
    p.k_min = o.k_min;
    p.k_max = o.k_max;
    p.tol = o.tol;
    p.zpts = reinterpret_cast<const double2 *>(z);
    p.gweight = weight;
    p.grad_z = reinterpret_cast<double2 *>(grad_z);
    p.grad_bands = reinterpret_cast<double2 *>(grad_bands);
    p.u_out = reinterpret_cast<double2 *>(u_out);
    p.v_out = reinterpret_cast<double2 *>(v_out);
    p.sigma = sigma;
    p.status = status;
    p.steps = steps;
    p.flags = reinterpret_cast<const int *>(ws + L.flags);
    p.counter = reinterpret_cast<int *>(ws + L.flags) + 1;
    p.q1 = reinterpret_cast<const double2 *>(ws + L.q1);
    p.wdata = ws + L.wdata;
    p.warp_bytes = L.warp_bytes;
    p.row_bytes = L.row_bytes;
    p.piv_offset = (2 * A->kl + A->ku + 1 + 4) * 512;
    p.trow = A->n;
    p.P = nwarps * 32;

    if (grad_bands &&
        cudaMemsetAsync(grad_bands, 0, sizeof(psa_c64) * (size_t)(A->kl + A->ku + 1) * (size_t)n, stream) != cudaSuccess)
        return PSA_ECUDA;
    k_start_vector<<<1, 256, 0, stream>>>(reinterpret_cast<double2 *>(ws + L.q1), A->n, o.seed);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    if (cudaMemsetAsync(ws + L.flags, 0, kAlign, stream) != cudaSuccess) return PSA_ECUDA;
    {
        const int64_t total = (int64_t)(A->kl + A->ku + 1) * A->n;
        const int64_t blocks = (total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024;
        k_check_finite<<<(unsigned)blocks, 256, 0, stream>>>(p.bands, A->n, A->kl, A->ku,
                                                              reinterpret_cast<int *>(ws + L.flags));
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    }
    if (n_pts == 0) return PSA_OK;
    if (ops.launch(p, stream) != cudaSuccess) return PSA_ECUDA;
    return PSA_OK;
}

}  // namespace
}  // namespace psa

extern "C" {

int psa_sigma_min_grad(const psa_band *A, const psa_c64 *z, int64_t n_pts, const double *weight, double *sigma,
                       psa_c64 *grad_z, psa_c64 *grad_bands, int8_t *status, int32_t *steps,
                       const psa_lanczos_opts *opts, void *workspace, size_t ws_bytes, void *stream_ptr)
{
    return sigma_min_grad_impl(A, z, n_pts, weight, sigma, grad_z, grad_bands, nullptr, nullptr, status, steps,
                               opts, workspace, ws_bytes, stream_ptr);
}

int psa_sigma_min_pairs(const psa_band *A, const psa_c64 *z, int64_t n_pts, double *sigma, psa_c64 *grad_z,
                        psa_c64 *u, psa_c64 *v, int8_t *status, int32_t *steps, const psa_lanczos_opts *opts,
                        void *workspace, size_t ws_bytes, void *stream_ptr)
{
    if (n_pts > 0 && (!u || !v)) return PSA_EINVAL;
    return sigma_min_grad_impl(A, z, n_pts, nullptr, sigma, grad_z, nullptr, n_pts > 0 ? u : nullptr, v, status,
                               steps, opts, workspace, ws_bytes, stream_ptr);
}

int psa_band_grad_from_pairs(const psa_band *A, int64_t n_pts, const psa_c64 *u, const psa_c64 *v,
                             const double *weight, psa_c64 *grad_bands, void *stream_ptr)
{
    if (!band_ok(A) || n_pts < 0 || !grad_bands || (n_pts > 0 && (!u || !v || !weight))) return PSA_EINVAL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    const int64_t nent = (int64_t)(A->kl + A->ku + 1) * A->n;
    if (n_pts == 0)
        return cudaMemsetAsync(grad_bands, 0, sizeof(psa_c64) * (size_t)nent, stream) == cudaSuccess ? PSA_OK
                                                                                                     : PSA_ECUDA;
    const int64_t blocks = (nent * 32 + 255) / 256 < 65536 ? (nent * 32 + 255) / 256 : 65536;
    k_band_grad_pairs<<<(unsigned)blocks, 256, 0, stream>>>(A->n, A->kl, A->ku, n_pts,
                                                            reinterpret_cast<const double2 *>(u),
                                                            reinterpret_cast<const double2 *>(v), weight,
                                                            reinterpret_cast<double2 *>(grad_bands));
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

// ------------------------------------------------------------------ batches

int psa_batch_plan_bytes(int32_t nmat, size_t *bytes)
{
    if (nmat < 0 || !bytes) return PSA_EINVAL;
    *bytes = kPlanMatOff + align_up(sizeof(PlanMat) * (size_t)nmat);
    return PSA_OK;
}

int psa_batch_plan(const psa_batch_entry *entries, int32_t nmat, void *plan, size_t plan_bytes)
{
    size_t need = 0;
    if (psa_batch_plan_bytes(nmat, &need) != PSA_OK || !plan || plan_bytes < need || (nmat > 0 && !entries))
        return PSA_EINVAL;
    for (int32_t m = 0; m < nmat; ++m) {
        const psa_batch_entry &e = entries[m];
        const psa_grid &g = e.g;
        if (!band_ok(&e.A) || !e.A.bands || e.out_offset < 0) return PSA_EINVAL;
        if (!(std::isfinite(g.re_min) && std::isfinite(g.re_max) && std::isfinite(g.im_min) &&
              std::isfinite(g.im_max)) ||
            g.re_min > g.re_max || g.im_min > g.im_max || g.nx < 1 || g.ny < 1 ||
            (int64_t)g.nx * g.ny > 2147483647LL)
            return PSA_EINVAL;
        if (e.A.kl > kMaxKL || e.A.ku > kMaxKU || !fits_row_offsets(&e.A)) return PSA_EUNSUPPORTED;
    }
    // matrices by class (kl, ku), within a class by decreasing n (stable)
    std::vector<int32_t> ord((size_t)nmat);
    for (int32_t m = 0; m < nmat; ++m) ord[(size_t)m] = m;
    auto cls = [&](int32_t m) { return entries[m].A.kl * (kMaxKU + 1) + entries[m].A.ku; };
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
        if (cls(a) != cls(b)) return cls(a) < cls(b);
        return entries[a].A.n > entries[b].A.n;
    });
    char *const base = static_cast<char *>(plan);
    std::memset(base, 0, need);
    PlanHeader &H = *reinterpret_cast<PlanHeader *>(base);
    PlanClass *const C = reinterpret_cast<PlanClass *>(base + kPlanClassOff);
    PlanMat *const M = reinterpret_cast<PlanMat *>(base + kPlanMatOff);
    int64_t q1 = 0;
    int nclass = 0;
    for (int32_t r = 0; r < nmat; ++r) {
        const psa_batch_entry &e = entries[ord[(size_t)r]];
        if (r == 0 || cls(ord[(size_t)r]) != cls(ord[(size_t)r - 1])) {
            PlanClass &c = C[nclass++];
            c.kl = e.A.kl;
            c.ku = e.A.ku;
            c.n_max = e.A.n;  // the class's first matrix is its largest
            c.first = r;
        }
        PlanClass &c = C[nclass - 1];
        PlanMat &pm = M[r];
        pm.bands = reinterpret_cast<const double2 *>(e.A.bands);
        pm.n = e.A.n;
        pm.nx = e.g.nx;
        pm.ny = e.g.ny;
        pm.re_min = e.g.re_min;
        pm.im_min = e.g.im_min;
        pm.hx = e.g.nx > 1 ? (e.g.re_max - e.g.re_min) / (double)(e.g.nx - 1) : 0.0;
        pm.hy = e.g.ny > 1 ? (e.g.im_max - e.g.im_min) / (double)(e.g.ny - 1) : 0.0;
        pm.out_off = e.out_offset;
        pm.q1_off = q1;
        pm.gstart = c.ngroups;
        pm.estart = c.nchunks;
        const int64_t groups = (int64_t)((e.g.nx + 7) / 8) * ((e.g.ny + 3) / 4);
        c.ngroups += groups;
        c.nchunks += (groups + 31) / 32;
        c.count += 1;
        q1 += e.A.n;
        if (c.ngroups > 2147483647LL) return PSA_EUNSUPPORTED;
        if (e.A.n > H.max_n) H.max_n = e.A.n;
    }
    for (int c = 0; c < nclass; ++c)
        if (C[c].ngroups > H.max_ngroups) H.max_ngroups = C[c].ngroups;
    H.magic = kPlanMagic;
    H.nmat = nmat;
    H.nclass = nclass;
    H.q1_total = q1;
    return PSA_OK;
}

namespace {

// Batch workspace: [class counters: 2 ints per class][mflags: one int per matrix]
// [start vectors][per stream: schedule of the largest class][per stream: region of
// warp blocks, used by the stream's classes one after another].
struct BatchLayout {
    size_t counters, mflags, q1, sched, regions;  // offsets
    size_t sched_bytes;                             // one stream's schedule
};

BatchLayout batch_layout(const PlanHeader &H, int nstreams)
{
    BatchLayout B{};
    size_t off = 0;
    B.counters = off; off += align_up(sizeof(int) * 2 * (size_t)kMaxClasses);
    B.mflags = off;   off += align_up(sizeof(int) * (size_t)(H.nmat > 0 ? H.nmat : 1));
    B.q1 = off;       off += align_up(sizeof(double2) * (size_t)H.q1_total);
    B.sched_bytes = sched_bytes(H.max_ngroups);
    B.sched = off;    off += (size_t)nstreams * B.sched_bytes;
    B.regions = off;
    return B;
}

bool plan_ok(const void *plan_host)
{
    if (!plan_host) return false;
    const PlanHeader &H = *static_cast<const PlanHeader *>(plan_host);
    return H.magic == kPlanMagic && H.nmat >= 0 && H.nclass >= 0 && H.nclass <= kMaxClasses &&
           (H.nmat == 0) == (H.nclass == 0);
}

const PlanClass *plan_classes(const void *plan_host)
{
    return reinterpret_cast<const PlanClass *>(static_cast<const char *>(plan_host) + kPlanClassOff);
}

// Estimated work of a class: sum over its matrices of points x n x flops per
// Lanczos row-step (the step count is not known before the run).
double class_cost(const void *plan_host, const PlanClass &c)
{
    const PlanMat *M = reinterpret_cast<const PlanMat *>(static_cast<const char *>(plan_host) + kPlanMatOff);
    double w = 0.0;
    for (int m = c.first; m < c.first + c.count; ++m)
        w += (double)M[m].nx * (double)M[m].ny * (double)M[m].n;
    return w * (16.0 * (2 * c.kl + c.ku) + 30.0);
}

// Classes in launch order (decreasing estimated work) and the stream of each:
// every class goes to the stream with the least estimated work so far (first on ties).
void stream_schedule(const void *plan_host, int nclass, int nstreams, int *order, int *lane)
{
    const PlanClass *C = plan_classes(plan_host);
    double cost[kMaxClasses];
    for (int c = 0; c < nclass; ++c) {
        order[c] = c;
        cost[c] = class_cost(plan_host, C[c]);
    }
    std::stable_sort(order, order + nclass, [&](int a, int b) { return cost[a] > cost[b]; });
    double load[kMaxStreams] = {};
    for (int r = 0; r < nclass; ++r) {
        const int c = order[r];
        int s = 0;
        for (int t = 1; t < nstreams; ++t)
            if (load[t] < load[s]) s = t;
        lane[c] = s;
        load[s] += cost[c];
    }
}

// Events per device: [0] forks the auxiliary streams off the caller's stream,
// [1 + k] joins auxiliary stream k back.
constexpr int kMaxDevices = 64;
std::mutex g_ev_mu;
cudaEvent_t g_ev[kMaxDevices][kMaxStreams] = {};

int batch_events(cudaEvent_t **ev)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PSA_ECUDA;
    std::lock_guard<std::mutex> lock(g_ev_mu);
    for (int k = 0; k < kMaxStreams; ++k)
        if (!g_ev[dev][k] && cudaEventCreateWithFlags(&g_ev[dev][k], cudaEventDisableTiming) != cudaSuccess) {
            g_ev[dev][k] = nullptr;
            return PSA_ECUDA;
        }
    *ev = g_ev[dev];
    return PSA_OK;
}

}  // namespace

int psa_batch_workspace_bytes(const void *plan_host, const psa_lanczos_opts *opts, int64_t points_in_flight,
                              int32_t n_streams, size_t *bytes)
{
    if (!plan_ok(plan_host) || points_in_flight < 1 || n_streams < 1 || n_streams > kMaxStreams || !bytes)
        return PSA_EINVAL;
    const psa_lanczos_opts o = opts ? *opts : psa_default_opts();
    if (!opts_ok(o)) return PSA_EINVAL;
    const PlanHeader &H = *static_cast<const PlanHeader *>(plan_host);
    const PlanClass *C = plan_classes(plan_host);
    const BatchLayout B = batch_layout(H, n_streams);
    size_t wmax = 0;
    for (int c = 0; c < H.nclass; ++c) {
        const int64_t nw_req = (points_in_flight + 31) / 32;
        const int64_t nw = nw_req < C[c].ngroups ? nw_req : C[c].ngroups;
        const size_t w = (size_t)nw * (size_t)layout(C[c].n_max, C[c].kl, C[c].ku, o.k_max, 1, 0).warp_bytes;
        if (w > wmax) wmax = w;
    }
    *bytes = B.regions + (size_t)n_streams * wmax;
    return PSA_OK;
}

int psa_sigma_min_batched(const void *plan_host, const void *plan_dev, const double *eps, int32_t n_eps,
                          double *sigma, uint32_t *mask, int8_t *status, int32_t *steps,
                          const psa_lanczos_opts *opts, int64_t points_in_flight, int32_t order, void *workspace,
                          size_t ws_bytes, void *stream_ptr, void *const *aux_streams, int32_t n_aux)
{
    if (!plan_ok(plan_host) || !plan_dev || (reinterpret_cast<uintptr_t>(plan_dev) % kAlign) != 0 || !sigma)
        return PSA_EINVAL;
    if (n_eps < 0 || n_eps > kMaxEps || (n_eps > 0 && !eps)) return PSA_EINVAL;
    for (int l = 0; l < n_eps; ++l)
        if (!std::isfinite(eps[l]) || !(eps[l] > 0.0)) return PSA_EINVAL;
    if (points_in_flight < 0 || order < PSA_BATCH_ORDER_AUTO || order > PSA_BATCH_ORDER_ESTIMATE) return PSA_EINVAL;
    if (n_aux < 0 || n_aux > kMaxStreams - 1 || (n_aux > 0 && !aux_streams)) return PSA_EINVAL;
    for (int k = 0; k < n_aux; ++k) {
        if (aux_streams[k] == stream_ptr) return PSA_EINVAL;
        for (int j = 0; j < k; ++j)
            if (aux_streams[j] == aux_streams[k]) return PSA_EINVAL;
    }
    const psa_lanczos_opts o = opts ? *opts : psa_default_opts();
    if (!opts_ok(o)) return PSA_EINVAL;
    const PlanHeader &H = *static_cast<const PlanHeader *>(plan_host);
    const PlanClass *C = plan_classes(plan_host);
    const PlanMat *Md = reinterpret_cast<const PlanMat *>(static_cast<const char *>(plan_dev) + kPlanMatOff);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return PSA_EWORKSPACE;
    if (H.nmat == 0) return PSA_OK;
    const int nstreams = 1 + n_aux;
    const BatchLayout B = batch_layout(H, nstreams);
    if (ws_bytes <= B.regions) return PSA_EWORKSPACE;
    const size_t region = (ws_bytes - B.regions) / (size_t)nstreams / kAlign * kAlign;

    // per class: kernel, warps in flight, stream and work-order decision, all checked
    // before anything is launched
    struct ClassRun {
        KernelOps ops;
        int64_t nwarps;
        bool ordered;
        Layout L;
    } run[kMaxClasses];
    for (int c = 0; c < H.nclass; ++c) {
        const PlanClass &pc = C[c];
        if (pc.kl < 0 || pc.kl > kMaxKL || pc.ku < 0 || pc.ku > kMaxKU || pc.count < 1 || pc.ngroups < 1 ||
            pc.first < 0 || pc.first + pc.count > H.nmat || pc.ngroups > H.max_ngroups)
            return PSA_EINVAL;
        if (pc.count > 65535) return PSA_EUNSUPPORTED;  // one grid row of the input check per matrix
        ClassRun &r = run[c];
        r.ops = pick_ops(pc.kl, pc.ku);
        if (!r.ops.launch) return PSA_EUNSUPPORTED;
        const Layout L1 = layout(pc.n_max, pc.kl, pc.ku, o.k_max, 1, 0);
        int64_t nw = (int64_t)(region / (size_t)L1.warp_bytes);
        if (nw < 1) return PSA_EWORKSPACE;
        int64_t full = 0;
        const int frc = full_threads(r.ops, &full);
        if (frc != PSA_OK) return frc;
        if (nw > full / 32) nw = full / 32;
        if (points_in_flight > 0 && nw > (points_in_flight + 31) / 32) nw = (points_in_flight + 31) / 32;
        if (nw > pc.ngroups) nw = pc.ngroups;
        if (nw >= 4) nw = round_down(nw, 4);
        r.nwarps = nw;
        r.ordered = order == PSA_BATCH_ORDER_ESTIMATE ? pc.ngroups > 1
                    : order == PSA_BATCH_ORDER_AUTO   ? pc.ngroups >= 2 * nw && pc.ngroups > 1
                                                      : false;
        r.L = L1;
    }
    int corder[kMaxClasses], lane[kMaxClasses];
    stream_schedule(plan_host, H.nclass, nstreams, corder, lane);
    cudaEvent_t *ev = nullptr;
    if (nstreams > 1) {
        const int erc = batch_events(&ev);
        if (erc != PSA_OK) return erc;
    }

    cudaStream_t streams[kMaxStreams] = {static_cast<cudaStream_t>(stream_ptr)};
    for (int k = 0; k < n_aux; ++k) streams[1 + k] = static_cast<cudaStream_t>(aux_streams[k]);
    char *ws = static_cast<char *>(workspace);
    int *const counters = reinterpret_cast<int *>(ws + B.counters);
    int *const mflags = reinterpret_cast<int *>(ws + B.mflags);
    double2 *const q1 = reinterpret_cast<double2 *>(ws + B.q1);

    if (cudaMemsetAsync(ws, 0, B.q1, streams[0]) != cudaSuccess) return PSA_ECUDA;  // counters and mflags
    k_batch_start_vectors<<<(unsigned)H.nmat, 256, 0, streams[0]>>>(Md, q1, o.seed);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    for (int c = 0; c < H.nclass; ++c) {
        const PlanClass &pc = C[c];
        const int64_t total = (int64_t)(pc.kl + pc.ku + 1) * pc.n_max;
        const int64_t bx = (total + 255) / 256 < 64 ? (total + 255) / 256 : 64;
        k_batch_check_finite<<<dim3((unsigned)bx, (unsigned)pc.count), 256, 0, streams[0]>>>(Md + pc.first, pc.kl,
                                                                                            pc.ku, mflags + pc.first);
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    }
    if (nstreams > 1) {
        if (cudaEventRecord(ev[0], streams[0]) != cudaSuccess) return PSA_ECUDA;
        for (int k = 1; k < nstreams; ++k)
            if (cudaStreamWaitEvent(streams[k], ev[0], 0) != cudaSuccess) return PSA_ECUDA;
    }

    for (int r_ = 0; r_ < H.nclass; ++r_) {
        const int c = corder[r_];
        const PlanClass &pc = C[c];
        const ClassRun &r = run[c];
        const int s = lane[c];
        cudaStream_t st = streams[s];
        int *const hist = reinterpret_cast<int *>(ws + B.sched + (size_t)s * B.sched_bytes);
        int *const cursor = hist + kBuckets;
        int *const bucket = cursor + kBuckets;
        int *const order_arr = bucket + H.max_ngroups;
        KParams p{};
        p.kl = pc.kl;
        p.ku = pc.ku;
        p.pmats = Md + pc.first;
        p.nmats = pc.count;
        p.trow = pc.n_max;
        p.mflags = mflags + pc.first;
        p.ngroups = pc.ngroups;
        p.nchunks = pc.nchunks;
        for (int l = 0; l < kMaxEps; ++l) p.eps[l] = l < n_eps ? eps[l] : 0.0;
        p.n_eps = n_eps;
        p.k_min = o.k_min;
        p.k_max = o.k_max;
        p.tol = o.tol;
        p.sigma = sigma;
        p.mask = mask;  // every point of a batch is evaluated and writes its bits
        p.status = status;
        p.steps = steps;
        p.flags = counters;
        p.counter = counters + 2 * c;
        p.estimate = 0;
        p.order = r.ordered ? order_arr : nullptr;
        p.sched_bucket = bucket;
        p.sched_hist = hist;
        p.q1 = q1;
        p.wdata = ws + B.regions + (size_t)s * region;
        p.warp_bytes = r.L.warp_bytes;
        p.row_bytes = r.L.row_bytes;
        p.piv_offset = (2 * pc.kl + pc.ku + 1 + 3) * 512;
        p.P = r.nwarps * 32;
        if (r.ordered) {
            if (cudaMemsetAsync(hist, 0, sizeof(int) * kBuckets, st) != cudaSuccess) return PSA_ECUDA;
            KParams pe = p;
            pe.estimate = 1;
            pe.order = nullptr;
            pe.k_min = pe.k_max = o.k_max < kEstimateSteps ? o.k_max : kEstimateSteps;
            pe.tol = 0.0;
            pe.counter = counters + 2 * c + 1;
            pe.sigma = nullptr;
            pe.mask = nullptr;
            pe.status = nullptr;
            pe.steps = nullptr;
            if (r.ops.launch(pe, st) != cudaSuccess) return PSA_ECUDA;
            k_sched_scan<<<1, kScanThreads, 0, st>>>(hist, cursor);
            if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
            const int64_t sb = (pc.ngroups + 255) / 256 < 4096 ? (pc.ngroups + 255) / 256 : 4096;
            k_sched_scatter<<<(unsigned)sb, 256, 0, st>>>(bucket, cursor, order_arr, pc.ngroups);
            if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
        }
        if (r.ops.launch(p, st) != cudaSuccess) return PSA_ECUDA;
    }
    for (int k = 1; k < nstreams; ++k) {
        if (cudaEventRecord(ev[k], streams[k]) != cudaSuccess) return PSA_ECUDA;
        if (cudaStreamWaitEvent(streams[0], ev[k], 0) != cudaSuccess) return PSA_ECUDA;
    }
    return PSA_OK;
}

int psa_probe_dfma_rate(int32_t iters, double *dfma_per_s, void *stream_ptr)
{
    if (iters < 1 || !dfma_per_s) return PSA_EINVAL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSA_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PSA_ECUDA;
    const int threads = 512, blocks = sms;  // 16 warps per SM
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PSA_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return PSA_ECUDA; }
    k_probe_dfma<<<blocks, threads, 0, stream>>>(64, 1.0000001, 1e-9);  // warm-up
    cudaEventRecord(e0, stream);
    k_probe_dfma<<<blocks, threads, 0, stream>>>(iters, 1.0000001, 1e-9);
    cudaEventRecord(e1, stream);
    int rc = PSA_OK;
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
        rc = PSA_ECUDA;
    else
        *dfma_per_s = (double)blocks * threads * 8.0 * (double)iters / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"
