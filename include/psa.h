/*
 * psa.h -- C ABI of the GB300 sigma_min grid engine (libpsa.so).
 *
 * The library evaluates sigma_min(zI - A), the smallest singular value of
 * zI - A, at the points z of a rectangular complex grid or of a list of grid
 * points, for a banded complex matrix A, and thresholds it at a list of
 * epsilon levels. This is the quantity whose level sets are the
 * epsilon-pseudospectra (paper Sec. 2, Definition "Pseudospectrum": the set
 * {z : sigma_min(zI - A) <= eps}), evaluated on the grid of Sec. 2.1 and, in
 * restricted mode, only on the predicted region R of the hybrid method
 * (Sec. 4: sigma_min is computed exactly for z in R and every other point is
 * classified non-sensitive).
 *
 * Method per point (hand-written CUDA for sm_103a, complex FP64 throughout):
 * B = zI - A is factored by banded Gaussian elimination with partial pivoting
 * (pivot = largest |Re| + |Im| in the column, first on ties; U gains kl
 * extra superdiagonals), then the Lanczos process on H = (B B^*)^{-1}, each
 * product formed by four banded triangular sweeps, gives
 * sigma_min = lambda_max(H)^{-1/2}. The paper computes the same quantity with a
 * dense SVD (Sec. 2.1); the banded path gives it in O(n (2kl+ku)) work per
 * Lanczos step instead of O(n^3).
 *
 * Conventions shared by every call:
 *  - All calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream); the library never synchronises the device and
 *    allocates no memory. The caller owns every buffer.
 *  - Device pointers must point to memory of the current CUDA device.
 *  - Return value: PSA_OK (0) or a negative PSA_E* code; psa_strerror()
 *    gives its text. On error nothing is launched.
 */
#ifndef PSA_H
#define PSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define PSA_OK 0
#define PSA_EINVAL (-1)      /* an argument is out of range or a required pointer is NULL */
#define PSA_EWORKSPACE (-2)  /* workspace too small (or NULL) for even one warp of points */
#define PSA_ECUDA (-3)       /* a CUDA launch or query failed (see cudaGetLastError) */
#define PSA_EUNSUPPORTED (-4) /* band widths beyond kl <= 4, ku <= 8 */
#define PSA_ESTATIC (-5)     /* psa_sigma_min_static: the problem needs more scratch than
                                PSA_STATIC_SCRATCH_BYTES for one warp (32 points) */

/* ----------------------------------------------------- per-point status */
#define PSA_PT_OK 0             /* converged (or fixed step count completed) */
#define PSA_PT_SINGULAR 1       /* exact zero pivot column: B singular, sigma = 0 */
#define PSA_PT_NOT_CONVERGED 2  /* k_max steps without meeting the stopping test */
#define PSA_PT_NONFINITE 3      /* A has a non-finite entry in its band: sigma = 0 */
#define PSA_PT_NOT_EVALUATED 4  /* restricted mode: point not in the list; sigma = NaN,
                                   mask = 0 (non-sensitive, paper Sec. 4) */
#define PSA_PT_UNDERFLOW 5      /* sigma_min below the double range (a solve overflowed,
                                   |(zI - A)^{-1}| > ~1e308): sigma reported as 0 */

/* Complex FP64, layout-identical to cuDoubleComplex and torch.complex128. */
typedef struct {
    double re, im;
} psa_c64;

/* Band matrix A of order n with kl subdiagonals and ku superdiagonals.
 * `bands` is a DEVICE pointer to (kl + ku + 1) * n values, diagonal-major:
 *   bands[(d + kl) * n + i] = A[i][i + d],  d in [-kl, ku], i in [0, n).
 * Entries with i + d outside [0, n) are never read. Read-only. */
typedef struct {
    int32_t n, kl, ku;
    const psa_c64 *bands;
} psa_band;

/* Grid of the complex plane (paper Sec. 2.1): nx abscissae and ny ordinates,
 *   x_j = fma(j, (re_max - re_min) / (nx - 1), re_min),  j in [0, nx)
 *   y_i = fma(i, (im_max - im_min) / (ny - 1), im_min),  i in [0, ny)
 * (a count of 1 gives the single value re_min / im_min). Point (i, j) is
 * z = x_j + i y_i, stored row-major at flat index i * nx + j (row = Im). */
typedef struct {
    double re_min, re_max, im_min, im_max;
    int32_t nx, ny;
} psa_grid;

/* Lanczos controls.
 *  k_min, k_max: minimum and maximum number of Lanczos steps, 1 <= k_max <= 65535,
 *                0 <= k_min <= k_max. k_min = k_max = k runs exactly k steps
 *                (unless the Krylov space is exhausted, beta = 0).
 *  tol:          stopping test after step j >= max(k_min, 2): stop when the top
 *                Ritz value moved by at most tol * theta_j,
 *                theta_j - theta_{j-1} <= tol * theta_j.  tol >= 0.
 *  seed:         start vector q_1 = h / |h|, h_i = u(2i) + i u(2i+1), u(c) the
 *                c-th SplitMix64 output for this seed mapped to [-1, 1).
 * psa_default_opts() gives k_min = 2, k_max = 1000, tol = 1e-13, seed = 0. */
typedef struct {
    int32_t k_min, k_max;
    double tol;
    uint64_t seed;
} psa_lanczos_opts;

/* Library version (major * 10000 + minor * 100 + patch). */
int psa_version(void);

/* Text of a PSA_* error code (static storage). */
const char *psa_strerror(int code);

/* Default Lanczos controls (converged mode). */
psa_lanczos_opts psa_default_opts(void);

/* Bytes of device workspace that psa_sigma_min needs to keep
 * `points_in_flight` points in flight at once (rounded up to whole warps of
 * 32), for calls of up to `npoints` points (grid points, or list entries in
 * restricted mode). The workspace holds a 256-byte flag block; the work-order
 * schedule (32 KB plus 8 bytes per group of 32 points, at most npoints / 8 + 2
 * groups); the shared start vector (n complex values); and one block per
 * warp: for each of the n rows the warp's pivoted band factor (2kl + ku + 1
 * complex values per point), three Lanczos vectors and the pivot offsets, then
 * the tridiagonal coefficients (2 * k_max values per point). With npoints = 0
 * the schedule is left out; psa_sigma_min then takes the groups in grid order,
 * with the same results but a longer tail. Host call, no device work.
 * Errors: PSA_EINVAL for bad A fields (bands pointer may be NULL here),
 * bad opts, points_in_flight < 1, npoints < 0 or bytes == NULL. */
int psa_workspace_bytes(const psa_band *A, const psa_lanczos_opts *opts,
                        int64_t points_in_flight, int64_t npoints, size_t *bytes);

/* Points in flight that fill the current device once with the kernel for
 * A's band shape (SM count x resident blocks x 128 threads, from the CUDA
 * occupancy calculator), capped at `npoints` rounded up to 32. Host call.
 * Errors: PSA_EINVAL (bad A fields, npoints < 1 or out == NULL),
 * PSA_EUNSUPPORTED, PSA_ECUDA. */
int psa_default_points_in_flight(const psa_band *A, int64_t npoints, int64_t *out);

/* sigma_min(zI - A) and its epsilon masks over a grid.
 *
 *  A        band matrix (device bands), 1 <= n, 0 <= kl, ku <= n - 1,
 *           kl <= 4, ku <= 8 and n * ((2kl + ku + 4) * 512 + 128) < 2^31
 *           (else PSA_EUNSUPPORTED).
 *  g        grid; finite bounds with re_min <= re_max, im_min <= im_max;
 *           nx, ny >= 1 and nx * ny <= 2^31 - 1.
 *  eps      HOST array of n_eps levels, 0 <= n_eps <= 32, each finite and > 0.
 *           Bit l of mask[p] is set iff sigma[p] <= eps[l] (inclusive, the
 *           sensitive zone of paper Sec. 2.1).
 *  idx      DEVICE array of n_idx flat grid indices (restricted mode, paper
 *           Sec. 4) or NULL for the full grid. Entries outside [0, nx*ny) are
 *           skipped. Points not listed get status PSA_PT_NOT_EVALUATED,
 *           sigma = NaN, mask = 0. A listed point gets bit-for-bit the value
 *           the full-grid call gives it (same per-point arithmetic).
 *  sigma    DEVICE output, nx * ny doubles (required).
 *  mask     DEVICE output, nx * ny uint32 (may be NULL).
 *  status   DEVICE output, nx * ny int8 PSA_PT_* codes (may be NULL).
 *  steps    DEVICE output, nx * ny int32 Lanczos steps taken (may be NULL).
 *  opts     Lanczos controls (NULL = psa_default_opts()).
 *  workspace, ws_bytes
 *           DEVICE scratch of ws_bytes bytes, 256-byte aligned; its size sets
 *           the number of points in flight (whole warps, at most one full
 *           occupancy of the device; see psa_workspace_bytes); it must not be
 *           used by another call that may run at the same time. Warps take
 *           groups of 32 points (8 x 4 grid tiles, or 32 list entries) from a
 *           counter in the workspace. When the workspace has room for the
 *           schedule, a short estimate pass (each group's anchor point, a few
 *           Lanczos steps) first orders the groups by decreasing sigma, which
 *           predicts the Lanczos step count, so the slowest groups start
 *           first. The assignment of points to warps varies between calls;
 *           every point's arithmetic, and so its result, does not.
 *  stream   cudaStream_t to launch on.
 * Errors: PSA_EINVAL, PSA_EWORKSPACE, PSA_EUNSUPPORTED, PSA_ECUDA. */
int psa_sigma_min(const psa_band *A, const psa_grid *g,
                  const double *eps, int32_t n_eps,
                  const int32_t *idx, int64_t n_idx,
                  double *sigma, uint32_t *mask, int8_t *status, int32_t *steps,
                  const psa_lanczos_opts *opts,
                  void *workspace, size_t ws_bytes, void *stream);

/* Bytes of device workspace for psa_sigma_min_grad with `points_in_flight`
 * points in flight (whole warps): like psa_workspace_bytes with a fourth vector
 * per row (the Ritz vector) and four tridiagonal arrays per point, no schedule.
 * Host call. Errors: PSA_EINVAL. */
int psa_grad_workspace_bytes(const psa_band *A, const psa_lanczos_opts *opts,
                             int64_t points_in_flight, size_t *bytes);

/* sigma_min(zI - A) and its adjoint gradients at n_pts explicit points z.
 *
 * For a simple smallest singular value with singular vectors u, v of
 * B = zI - A (B v = sigma u), d sigma = Re(u^* dB v), so
 *   grad_z[p]  = d sigma_p / d Re z + i d sigma_p / d Im z = conj(u^* v),
 *   grad_bands = sum_p weight[p] (d sigma_p / d Re a + i d sigma_p / d Im a)
 *              = -sum_p weight[p] u_i conj(v_{i+d})  for a = A[i][i+d],
 * in band storage (bands[(d + kl) * n + i]). These are the derivatives that the
 * Newton refinement of eps-contours (paper Sec. 2, Definition "Pseudospectrum")
 * and a torch.autograd backward need. u is the Ritz vector of the converged
 * Lanczos process (a second pass replays the recurrence), v = B^{-1} u / |B^{-1} u|.
 *
 *  A, opts        as psa_sigma_min (kl <= 4, ku <= 8).
 *  z              DEVICE, n_pts complex points (any, not only grid points).
 *  weight         DEVICE, n_pts upstream weights; required when grad_bands != NULL.
 *  sigma          DEVICE output, n_pts doubles (required if n_pts > 0).
 *  grad_z         DEVICE output, n_pts complex (may be NULL). 0 where status is
 *                 not OK / NOT_CONVERGED or sigma = 0.
 *  grad_bands     DEVICE output, (kl + ku + 1) * n complex, zeroed and then summed
 *                 into (may be NULL; the sum's order varies between runs).
 *  status, steps  DEVICE outputs per point (may be NULL), codes as psa_sigma_min.
 *  workspace      DEVICE scratch, 256-byte aligned, of ws_bytes (psa_grad_workspace_bytes).
 * Asynchronous on `stream`; allocates nothing.
 * Errors: PSA_EINVAL, PSA_EWORKSPACE, PSA_EUNSUPPORTED, PSA_ECUDA. */
int psa_sigma_min_grad(const psa_band *A, const psa_c64 *z, int64_t n_pts, const double *weight,
                       double *sigma, psa_c64 *grad_z, psa_c64 *grad_bands,
                       int8_t *status, int32_t *steps, const psa_lanczos_opts *opts,
                       void *workspace, size_t ws_bytes, void *stream);

/* psa_sigma_min_grad without the band gradient, writing instead the singular
 * pair of every point, element-major: u[i * n_pts + p] and v[i * n_pts + p]
 * (DEVICE, n * n_pts complex each; B v = sigma u, |u| = |v| = 1, the phases
 * those of the kernel's Ritz vector; zeros where grad_z is 0). A backward pass
 * that learns its weights later then needs only psa_band_grad_from_pairs.
 * Other arguments and errors as psa_sigma_min_grad. */
int psa_sigma_min_pairs(const psa_band *A, const psa_c64 *z, int64_t n_pts, double *sigma, psa_c64 *grad_z,
                        psa_c64 *u, psa_c64 *v, int8_t *status, int32_t *steps, const psa_lanczos_opts *opts,
                        void *workspace, size_t ws_bytes, void *stream);

/* grad_bands[(d + kl) * n + i] = -sum_p weight[p] u_p[i] conj(v_p[i + d]), the
 * weighted band gradient of psa_sigma_min_grad, from stored singular pairs
 * (layout of psa_sigma_min_pairs; A's bands pointer is not read). One warp per
 * band entry with a fixed-order sum: the same bits on every run. DEVICE
 * pointers; asynchronous on stream. Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_band_grad_from_pairs(const psa_band *A, int64_t n_pts, const psa_c64 *u, const psa_c64 *v,
                             const double *weight, psa_c64 *grad_bands, void *stream);

/* Newton refinement of eps-contour crossings along grid rows (the level set
 * sigma_min(zI - A) = eps of paper Sec. 2, Definition "Pseudospectrum", on the
 * grid lines of Sec. 2.1). A crossing c of row rows[c] lies between columns
 * cols[c] and cols[c] + 1, where sigma - eps changes sign (s_lo, s_hi: sigma at
 * the two grid points). psa_contour_init sets the bracket lo, hi, the ordinate
 * y, the sign of f = sigma - eps at the left end (flo_neg), the first iterate x
 * (log sigma interpolated between the ends, kept within [0.05, 0.95] of the
 * bracket) and z = x + i y; done = 0, resid = inf. psa_contour_step takes sigma
 * and grad_z of psa_sigma_min_grad at z for the running crossings idx[0 .. na)
 * (sigma[a], grad_z[a] belong to crossing idx[a]) and, per crossing: resid =
 * |f| / eps, done when resid <= rtol or the bracket is narrower than 4 ulp;
 * the bracket end whose sign f has moves to x; the next x is the Newton step
 * x - f / (d sigma / d Re z) if it stays inside the bracket, else the
 * bracket's midpoint; z is updated. All arrays DEVICE, m (or na) entries;
 * asynchronous on stream. Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_contour_init(int32_t m, const int32_t *rows, const int32_t *cols, const psa_grid *g, const double *s_lo,
                     const double *s_hi, double eps, double *x, double *lo, double *hi, double *y, uint8_t *flo_neg,
                     uint8_t *done, double *resid, psa_c64 *z, void *stream);
int psa_contour_step(int32_t na, const int32_t *idx, const double *sigma, const psa_c64 *grad_z, double eps,
                     double rtol, double *x, double *lo, double *hi, const double *y, const uint8_t *flo_neg,
                     uint8_t *done, double *resid, psa_c64 *z, void *stream);

/* Size of the fixed device scratch used by psa_sigma_min_static (64 MiB). */
#define PSA_STATIC_SCRATCH_BYTES (64u << 20)

/* psa_sigma_min for callers that cannot allocate device memory. The paper
 * has no counterpart: this is a deployment variant of psa_sigma_min.
 *
 * Some callers cannot call cudaMalloc or any allocating routine: a host that
 * hands its GPU memory out once at start-up, a real-time or latency-bound
 * loop where allocation may block, a sandboxed plugin without allocator
 * rights. This entry point takes the same arguments as psa_sigma_min except
 * the workspace: its scratch is one file-scope device array of
 * PSA_STATIC_SCRATCH_BYTES (64 MiB) inside the library, which every GPU that
 * loads the library holds until the process exits. It allocates nothing and
 * calls no allocating routine; outputs and inputs remain the caller's.
 *
 *  - Set-up: every call looks up the array's device address on the current
 *    device (cudaGetSymbolAddress, no allocation), so the address stays right
 *    after cudaDeviceReset. The first call on a device may load the library's
 *    device code into its context; make that first call before any stream
 *    capture.
 *  - Size limit: the scratch must hold at least one warp of points (see
 *    psa_workspace_bytes with points_in_flight = 32); larger problems are
 *    rejected with PSA_ESTATIC and nothing is launched. Within the limit the
 *    number of points in flight is what fits, so big problems run slower
 *    than with a large caller workspace.
 *  - Sharing: every call uses the same array, which keeps the previous
 *    call's contents (each call clears the parts that must start at zero).
 *    Calls whose kernels may overlap on the GPU (different streams, or
 *    several host threads) race on the array: serialise them.
 * Results are bitwise those of psa_sigma_min on the same arguments (a point's
 * arithmetic does not depend on how many points are in flight).
 * Errors: the argument codes of psa_sigma_min (PSA_EINVAL, PSA_EUNSUPPORTED)
 * first, then PSA_ESTATIC, then PSA_ECUDA. */
int psa_sigma_min_static(const psa_band *A, const psa_grid *g,
                         const double *eps, int32_t n_eps,
                         const int32_t *idx, int64_t n_idx,
                         double *sigma, uint32_t *mask, int8_t *status, int32_t *steps,
                         const psa_lanczos_opts *opts, void *stream);

/* ------------------------------------------------------------------ batches
 * Many independent matrices, each with its own grid, in one call. The paper
 * evaluates one matrix at a time; a batch serves the same per-point quantity
 * to callers with many small or mid-size problems (a parameter sweep, a
 * family of discretisations), where one grid alone cannot fill the device.
 * Results are bit-identical to psa_sigma_min on each matrix alone with the
 * same opts: every point is computed by the same arithmetic from the same
 * start vector; only the order in which warps take the points differs. */

/* One matrix of a batch: its band (DEVICE bands pointer), its full grid, and
 * where its results start in the batch outputs: point (i, j) of the grid goes
 * to sigma[out_offset + i * g.nx + j] (likewise mask, status, steps). The
 * caller keeps the output ranges of different entries disjoint. */
typedef struct {
    psa_band A;
    psa_grid g;
    int64_t out_offset;
} psa_batch_entry;

/* Order of the groups (8 x 4 grid tiles) within one band-shape class. */
#define PSA_BATCH_ORDER_AUTO 0      /* estimate pass when warps take >= 2 groups each */
#define PSA_BATCH_ORDER_PLAN 1      /* plan order: matrices by decreasing n, tiles in grid order */
#define PSA_BATCH_ORDER_ESTIMATE 2  /* always: anchor points, 4 Lanczos steps, longest first */

/* Bytes of the plan of a batch of nmat matrices (host call). Errors: PSA_EINVAL
 * (nmat < 0 or bytes == NULL). */
int psa_batch_plan_bytes(int32_t nmat, size_t *bytes);

/* Builds the plan of a batch in HOST memory `plan` (plan_bytes from
 * psa_batch_plan_bytes): the matrices grouped into classes of equal (kl, ku),
 * each class ordered by decreasing n, with the offsets of each matrix's tiles,
 * start vector and outputs. The plan holds the entries' device bands pointers;
 * the caller copies its bytes unchanged to device memory (256-byte aligned)
 * before psa_sigma_min_batched and keeps both copies and the bands alive while
 * calls that use them run. Host call, no device work.
 * Errors: PSA_EINVAL (an entry with bad band or grid fields, a NULL bands
 * pointer, out_offset < 0, a grid of more than 2^31 - 1 points, nmat < 0,
 * plan NULL or plan_bytes too small), PSA_EUNSUPPORTED (kl > 4 or ku > 8, or
 * a class of more than 2^31 - 1 groups). */
int psa_batch_plan(const psa_batch_entry *entries, int32_t nmat, void *plan, size_t plan_bytes);

/* Bytes of device workspace for psa_sigma_min_batched with up to
 * `points_in_flight` points (whole warps) in flight in each class and
 * `n_streams` (1 to 8) streams: a counter block, one flag per matrix, the start
 * vectors of all matrices, then per stream the work-order schedule of the
 * largest class and a region of warp blocks (per warp the block
 * psa_workspace_bytes describes, for the largest n of the class) that the
 * classes of that stream use one after another. Host call.
 * Errors: PSA_EINVAL. */
int psa_batch_workspace_bytes(const void *plan_host, const psa_lanczos_opts *opts, int64_t points_in_flight,
                              int32_t n_streams, size_t *bytes);

/* sigma_min on every grid point of every matrix of a batch, with the eps
 * masks of psa_sigma_min. A set-up pass (all start vectors, input checks) on
 * `stream`, then per band-shape class an optional estimate pass and one
 * persistent sigma_min launch. With auxiliary streams the classes are split
 * over `stream` and the n_aux streams `aux_streams` (longest estimated first,
 * each class to the stream with the least estimated work so far; estimate =
 * points x n x flops per Lanczos row-step): the launches of several classes
 * are then in flight at once and the device's block scheduler fills the tail
 * of one class with blocks of the others. The auxiliary streams wait for the
 * set-up on `stream`, and `stream` waits for the last class of every auxiliary
 * stream before the call returns (events of the library, created at the first
 * call on a device). The call allocates no memory and copies nothing between
 * host and device, so a whole batch can be captured in one CUDA graph and
 * replayed (make one call outside capture first so that the events exist).
 *  plan_host, plan_dev  the plan (psa_batch_plan) in host memory and its copy
 *                   in device memory.
 *  eps, n_eps       as psa_sigma_min (host array).
 *  sigma, mask, status, steps  DEVICE outputs indexed by the entries'
 *                   out_offset (mask, status, steps may be NULL).
 *  opts             Lanczos controls (NULL = psa_default_opts()).
 *  points_in_flight per class at most this many points in flight (0: as many
 *                   as the workspace and one full occupancy of the device allow).
 *  order            PSA_BATCH_ORDER_*.
 *  workspace, ws_bytes  DEVICE scratch, 256-byte aligned
 *                   (psa_batch_workspace_bytes with the same number of
 *                   streams); each stream's region is (ws_bytes - fixed part)
 *                   / streams, and a class runs as many warps as its region
 *                   holds, up to the caps above.
 *  stream           cudaStream_t of the call.
 *  aux_streams, n_aux  0 to 7 further cudaStream_t, all different from each
 *                   other and from stream (n_aux = 0: every class on stream).
 * Errors: PSA_EINVAL (bad eps, opts or order, a plan whose header does not
 * check, n_aux out of range, a repeated stream), PSA_EUNSUPPORTED (a class of
 * more than 65535 matrices), PSA_EWORKSPACE (no room for one warp in some
 * class), PSA_ECUDA. */
int psa_sigma_min_batched(const void *plan_host, const void *plan_dev, const double *eps, int32_t n_eps,
                          double *sigma, uint32_t *mask, int8_t *status, int32_t *steps,
                          const psa_lanczos_opts *opts, int64_t points_in_flight, int32_t order,
                          void *workspace, size_t ws_bytes, void *stream, void *const *aux_streams,
                          int32_t n_aux);

/* --------------------------------------------------------------- classifier
 * The learned restriction of the hybrid method (paper Sec. 3-4): a network maps
 * per-point features to the probability that the point is sensitive; only the
 * points it selects get the exact sigma_min evaluation. Here the network is a
 * multilayer perceptron IN -> 256 -> 256 -> 256 -> 1 (SiLU hidden units,
 * sigmoid output) whose dense layers run as BF16 GEMMs on the tensor cores
 * with FP32 accumulation; training minimises binary cross-entropy with Adam
 * (Sec. 3.4). Parameters are one float32 vector theta (device) laid out as
 * W1[256][IN], b1[256], W2[256][256], b2[256], W3[256][256], b3[256],
 * w4[256], b4 (W[out][in], row-major). Features are BF16 rows of IN values
 * (the feature kernels of psa_features.cu fill them). */
#define PSA_MLP_IN 128
#define PSA_MLP_HIDDEN 256
#define PSA_MLP_PARAMS 164865

/* C[M][N] (float32, row-major, leading dimension ldc) = A[M][K] * B[N][K]^T
 * with A and B BF16 (raw uint16 bits) row-major, K contiguous, on the tensor
 * cores (FP32 accumulation). Device pointers, 16-byte aligned; N a multiple
 * of 128, K a multiple of 64, lda and ldb multiples of 8; M any.
 * Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int32_t M, int32_t N, int32_t K,
                  float *C, int64_t ldc, void *stream);

/* The paper's dual-path network (Sec. 3.2.2) on the same feature rows: a
 * coordinate pathway on the Fourier columns [0, 26) (26 -> 64 -> 64, Eq. for
 * h_c^(1), h_c^(2)), a matrix pathway on the feature columns [26, 61) (35 ->
 * 128 -> 64; the paper has 33 features, this library's set is listed at
 * psa_point_features), concatenation (128), the residual block h4 =
 * SiLU(W4 h3 + b4), h5 = SiLU(W5 h4 + b5), h6 = h4 + h5 (128), h7 =
 * SiLU(W7 h6 + b7) (64) and p = sigmoid(w . h7 + b). theta (DEVICE float32
 * [PSA_DUAL_PARAMS]) stores fused, padded matrices [out][in], row-major:
 *   WA[256][128], bA[256]: rows 0..63 = (W_c1, b_c1) on columns 0..25, rows
 *     64..191 = (W_m1, b_m1) on columns 26..60, all else zero;
 *   WB[128][256], bB[128]: rows 0..63 = W_c2 on columns 0..63, rows 64..127 =
 *     W_m2 on columns 64..191 (so WB's output is [h_c2 | h_m2] = h3);
 *   W4[128][128], b4, W5[128][128], b5;
 *   W7[128][128], b7[128]: rows 0..63 = (W7, b7), rows 64..127 zero;
 *   w[128] (entries 64..127 zero), b.
 * The zero entries are structural: training masks their gradients, so they
 * stay zero and the network has PSA_DUAL_TRAINABLE parameters. Same calling
 * conventions, batching, asynchrony and errors as psa_mlp_*. */
#define PSA_DUAL_PARAMS 115585
#define PSA_DUAL_TRAINABLE 60097
int psa_dual_workspace_bytes(int64_t rows, int32_t training, size_t *bytes);
int psa_dual_forward(const float *theta, const uint16_t *x, int64_t rows, float *prob, void *workspace,
                     size_t ws_bytes, void *stream);
int psa_dual_train_step(float *theta, float *adam_m, float *adam_v, int32_t step, float lr, const uint16_t *x,
                        const float *y, int64_t rows, float *loss, void *workspace, size_t ws_bytes, void *stream);

/* Number of GEMM tiles (of psa_gemm_bf16, psa_mlp_* and psa_dual_* on the
 * current device) whose bounded waits for a tensor-
 * memory copy or a tensor-core commit ran out since the previous call, then
 * reset to zero. A tile that times out writes NaN in place of its outputs (the
 * outputs of that call are undefined), waits once more for the work it issued,
 * frees its tensor memory and exits; the asynchronous calls themselves still
 * return PSA_OK. SYNCHRONISES the device (it reads a device counter); call it
 * where a result is read back anyway. The paper has no counterpart.
 * Errors: PSA_EINVAL (count NULL), PSA_ECUDA. */
int psa_mlp_timeouts(uint32_t *count);

/* Bytes of device workspace for psa_mlp_forward over `rows` rows (training = 0;
 * rows beyond 131072 are processed in passes of 131072) or for
 * psa_mlp_train_step on batches of `rows` rows (training = 1). Host call.
 * Errors: PSA_EINVAL. */
int psa_mlp_workspace_bytes(int64_t rows, int32_t training, size_t *bytes);

/* prob[r] = network(x[r]) for r < rows: x DEVICE BF16 [rows][IN] (16-byte
 * aligned), prob DEVICE float32 [rows], theta DEVICE float32
 * [PSA_MLP_PARAMS]; workspace DEVICE, 256-byte aligned, of ws_bytes >=
 * psa_mlp_workspace_bytes(rows, 0). Asynchronous on stream.
 * Errors: PSA_EINVAL, PSA_EWORKSPACE, PSA_ECUDA. */
int psa_mlp_forward(const float *theta, const uint16_t *x, int64_t rows, float *prob, void *workspace,
                    size_t ws_bytes, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, epsilon 1e-8, bias-corrected with the
 * 1-based step number `step`, learning rate lr) on the mean binary
 * cross-entropy of a batch: x DEVICE BF16 [rows][IN], y DEVICE float32 labels
 * in [0, 1]; theta, adam_m, adam_v DEVICE float32 [PSA_MLP_PARAMS] updated in
 * place; *loss (DEVICE float32) receives the batch's mean loss before the
 * step. rows a multiple of 128. Asynchronous on stream; no allocation, so a
 * step can be captured in a CUDA graph (step and lr are then fixed at capture).
 * Errors: PSA_EINVAL, PSA_EWORKSPACE, PSA_ECUDA. */
int psa_mlp_train_step(float *theta, float *adam_m, float *adam_v, int32_t step, float lr, const uint16_t *x,
                       const float *y, int64_t rows, float *loss, void *workspace, size_t ws_bytes, void *stream);

/* Classifier features (paper Sec. 3.1, 3.2.1). psa_matrix_stats reduces A's
 * band (one block, FP64) to the statistics below and samples the symbol
 * f(t) = sum_d abar_d e^{i d t} of the diagonal means abar_d at
 * PSA_SYMBOL_SAMPLES points t_k = 2 pi k / PSA_SYMBOL_SAMPLES (DEVICE outputs
 * stats[PSA_STATS], symbol[PSA_SYMBOL_SAMPLES]). The symbol curve stands in
 * for the eigenvalue set of the paper's eigenvalue features; the centroid
 * trace(A) / n is the eigenvalue centroid exactly. */
#define PSA_SYMBOL_SAMPLES 256
#define PSA_MAX_BAND 13
#define PSA_STATS 24
#define PSA_STAT_CEN_RE 0      /* Re, Im of trace(A) / n */
#define PSA_STAT_CEN_IM 1
#define PSA_STAT_RADIUS 2      /* max_k |f(t_k) - centroid| */
#define PSA_STAT_FRO 3         /* |A|_F */
#define PSA_STAT_NORM1 4       /* |A|_1 */
#define PSA_STAT_NORMINF 5     /* |A|_inf */
#define PSA_STAT_ASYM 6        /* |A - A^T|_F */
#define PSA_STAT_AHERM 7       /* |A - A^H|_F */
#define PSA_STAT_DIAG_MEAN 8   /* mean, std of |A_ii| */
#define PSA_STAT_DIAG_STD 9
#define PSA_STAT_OFF_MEAN 10   /* mean, std of |A_ij| over the other in-band positions */
#define PSA_STAT_OFF_STD 11
#define PSA_STAT_NNZ 12        /* entries with |A_ij| > 1e-10 */
#define PSA_STAT_SYM_RE_MEAN 13 /* mean, std, min, max of Re (f - centroid) */
#define PSA_STAT_SYM_RE_STD 14
#define PSA_STAT_SYM_RE_MIN 15
#define PSA_STAT_SYM_RE_MAX 16
#define PSA_STAT_SYM_IM_MEAN 17 /* the same for Im */
#define PSA_STAT_SYM_IM_STD 18
#define PSA_STAT_SYM_IM_MIN 19
#define PSA_STAT_SYM_IM_MAX 20
#define PSA_STAT_SYM_RMIN 21    /* min_k |f(t_k) - centroid| */
#define PSA_STAT_N 22
#define PSA_STAT_BAND 23        /* 16 kl + ku */
#define PSA_GLOBAL_FEATURES 28

/* A DEVICE band (kl + ku + 1 <= PSA_MAX_BAND). Errors: PSA_EINVAL,
 * PSA_EUNSUPPORTED, PSA_ECUDA. */
int psa_matrix_stats(const psa_band *A, double *stats, psa_c64 *symbol, void *stream);

/* Global feature vector (DEVICE float32 [PSA_GLOBAL_FEATURES]) from the
 * statistics and sigma4 (DEVICE): sigma_min(zI - A) at z = 0 and at the
 * centroid + 0.5, + 1, + 2 (the resolvent norms of Table 3 are 1 / sigma_min
 * exactly), for the level eps. Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_global_features(const double *stats, const double *sigma4, double eps, float *global, void *stream);

/* One BF16 row of PSA_MLP_IN features per point of the grid (idx NULL) or of
 * the flat grid indices idx[0 .. n_idx) (DEVICE), written to x (DEVICE,
 * 16-byte aligned) in point order: [0, 26) the Fourier encoding [c, sin 2^k c,
 * cos 2^k c], k = 1..6, of the grid coordinates c scaled to [-1, 1]^2;
 * 26..28 the distances g1 (to the closed polyline through the symbol samples),
 * g2 (to the centroid), g3 (mean distance to the samples), in units of the
 * symbol radius; 29, 30 log10 of g1 and g3; 31 the winding number of the
 * symbol curve about the point; [32, 32 + PSA_GLOBAL_FEATURES) the global
 * features; 32 + PSA_GLOBAL_FEATURES: log10 of the distance to the polyline
 * over eps; zeros after.
 * Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_point_features(const psa_grid *g, const int32_t *idx, int64_t n_idx, const double *stats,
                       const psa_c64 *symbol, const float *global, uint16_t *x, void *stream);

/* The paper's own spectrum features (Sec. 3.1, Table "matrix", f1 .. f10)
 * from a point set instead of the symbol curve: set[0 .. m) (DEVICE) is, for
 * example, the eigenvalues of A computed by a dense eigensolver. Overwrites in
 * stats (DEVICE, as written by psa_matrix_stats, whose centroid it keeps) the
 * radius R = max |set - centroid| and the entries PSA_STAT_SYM_RE_MEAN ..
 * PSA_STAT_SYM_RMIN with the mean, standard deviation, minimum and maximum of
 * Re and Im of (set - centroid) and min |set - centroid|; call
 * psa_global_features afterwards. Errors: PSA_EINVAL (m < 1, NULL), PSA_ECUDA. */
int psa_point_set_stats(const psa_c64 *set, int32_t m, double *stats, void *stream);

/* psa_point_features over any set of m >= 1 points (DEVICE set[0 .. m)).
 * closed = 1: the set is a closed polyline set[0] -> .. -> set[m - 1] -> set[0]
 * (psa_point_features is this with the PSA_SYMBOL_SAMPLES symbol samples);
 * closed = 0: the set is a point set such as the eigenvalues, and g1 is the
 * distance to its nearest point (Eq. (dist)), g3 the mean distance to its
 * points and column 31 (the winding number) is 0. Distances are in units of
 * stats' radius. Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_point_features_set(const psa_grid *g, const int32_t *idx, int64_t n_idx, const double *stats,
                           const psa_c64 *set, int32_t m, int32_t closed, const float *global, uint16_t *x,
                           void *stream);

/* Predicted region of the hybrid method (paper Sec. 3.6 and 4): mask[f] = 1
 * when some grid point within `radius` rows and columns of f (a box of
 * (2 radius + 1)^2 points, clipped to the grid) has prob >= tau. prob and
 * mask DEVICE, nx * ny entries. Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_region(const float *prob, float tau, int32_t nx, int32_t ny, int32_t radius, uint8_t *mask, void *stream);

/* The points of a mask in the sigma_min kernel's full-grid work order (8 x 4
 * tiles): slot[32 t + l] = flat index of lane l's point of tile t when it is
 * in the mask, else -1 (slot DEVICE, ceil(nx / 8) * ceil(ny / 4) * 32
 * entries). The non-negative entries, in order, are a restricted point list
 * whose chunks of 32 are compact patches of the grid.
 * Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_tile_slots(const uint8_t *mask, int32_t nx, int32_t ny, int32_t *slot, void *stream);

/* Measured FP64 throughput of this device: runs a kernel of independent DFMA
 * chains (iters iterations, 8 chains, SM count x 16 warps) on `stream`,
 * synchronises it and returns the rate in DFMA lane-operations per second in
 * *dfma_per_s. Used for the roofline of the FP64-bound path.
 * Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_probe_dfma_rate(int32_t iters, double *dfma_per_s, void *stream);

/* FP64 micro-benchmark behind the roofline and the one-lane-per-point layout:
 * one block of warps_per_sm (1..32) warps per SM; in each warp the first
 * active_lanes (1..32) lanes run `chains` (1 or 8) independent chains of `iters`
 * (1..2^24) operations `op`: 0 DFMA, 1 DADD, 2 DMUL, 3 division, 4 square root.
 * Runs a warm-up and a timed launch on `stream`, synchronises, and returns
 * lane-operations per second (SMs x warps x active lanes x chains x iters /
 * time) in *lane_ops_per_s. Errors: PSA_EINVAL, PSA_ECUDA. */
int psa_probe_fp64(int32_t op, int32_t warps_per_sm, int32_t active_lanes, int32_t chains, int32_t iters,
                   double *lane_ops_per_s, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PSA_H */
