// psa_kernel.cuh -- the sigma_min(zI - A) kernel for one compile-time band shape.
//
// One thread evaluates one grid point; the 32 lanes of a warp hold 32
// neighbouring points of the grid and run the same instruction stream (same
// n, kl, ku), so every FP64 instruction does 32 lanes of useful work until a
// lane's Lanczos process stops. FP64 is the bound on GB300 (about 2 DFMA per
// SM per clock against 128 FFMA), so the code is arranged to issue as few
// FP64 instructions per point as the method allows:
//   * complex multiply-adds are written as 4 explicit fused multiply-adds;
//   * pivot comparisons, scale exponents and the Sturm sign test use integer
//     operations on the bit patterns;
//   * the reciprocal of each pivot is formed once in the factorisation, so the
//     solves multiply instead of divide;
//   * the Lanczos dot products and vector updates ride along the triangular
//     sweeps that produce their operands (four sweeps per step, no extra pass).
//
// Per point (paper Sec. 2.1: sigma_min(z) = sigma_n(zI - A); Sec. 2,
// Definition "Pseudospectrum"):
//   1. B = zI - A is factored by Gaussian elimination with partial pivoting
//      inside the band (pivot = largest |Re| + |Im| of rows j..j+kl, first on
//      ties), with a (kl+1) x (kl+ku+1) register window sliding down the band.
//   2. Lanczos on H' = (B B^*)^{-1} / 2^(2 e1): step k solves B x = v_k
//      (interchanges + L forward, U backward), solves B^* y = x (U^* forward,
//      L^* backward + interchanges), and forms w_k (proportional to
//      H' q_k - beta_{k-1} q_{k-1}), alpha_k = Re <q_k, H' q_k - ...>, and
//      in the next step's first sweep v_{k+1} (proportional to
//      u_{k+1} = w_k - alpha_k q_k) and beta_k = |u_{k+1}|. The stored vectors
//      keep a fixed power-of-two scale, so no sweep normalises them.
//   3. theta_k = lambda_max(T_k) by Newton's method on the characteristic
//      polynomial of T_k from above (monotone, warm-started at the previous
//      Ritz value); stop when theta_k - theta_{k-1} <= tol * theta_k, at
//      beta_k = 0 or at k_max. sigma = 2^(-e1) / sqrt(theta_k). A value that
//      leaves the double range (|B^{-1}| > ~1e308) ends the point with
//      status UNDERFLOW and sigma = 0.
//   4. Mask bit l = (sigma <= eps_l) (paper Sec. 2.1, Eq. (sensitive_zone)).
//
// Work distribution: each warp takes groups of 32 points from an atomic
// counter until the points run out, so warps that meet fast-converging points
// take more of them. On the full grid a group is an 8 x 4 tile of the grid
// (neighbouring points converge in similar step counts, so fewer lanes idle
// than with 32 points of one grid row); in restricted mode it is 32
// consecutive entries of the list. A short estimate pass (one anchor point per
// group, a few Lanczos steps) lets the groups be taken longest first, so the
// launch does not end on a few slow groups. Each warp owns one contiguous
// workspace block. In a batch launch (one band shape, many matrices) a group is a
// tile of one of the matrices: the warp finds the matrix by a binary search in the
// device plan, and its workspace block is sized for the largest matrix.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "psa_internal.h"

namespace psa {
namespace dev {

// ------------------------------------------------------------ complex FP64
// acc - a * b
__device__ __forceinline__ double2 c_sub_mul(double2 acc, double2 a, double2 b)
{
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
// acc - conj(a) * b
__device__ __forceinline__ double2 c_sub_conjmul(double2 acc, double2 a, double2 b)
{
    return make_double2(fma(-a.x, b.x, fma(-a.y, b.y, acc.x)), fma(-a.x, b.y, fma(a.y, b.x, acc.y)));
}
// a * b
__device__ __forceinline__ double2 c_mul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 c_mul_conj(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -(a.x * b.y)));
}

// Bit-pattern helpers (integer pipe).
__device__ __forceinline__ unsigned long long abs_bits(double d)
{
    return static_cast<unsigned long long>(__double_as_longlong(d)) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ int exp_field(double d) { return (__double2hiint(d) >> 20) & 0x7ff; }
// 2^e for e in [-1022, 1023], exact.
__device__ __forceinline__ double pow2i(int e) { return __hiloint2double((e + 1023) << 20, 0); }
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
// v * 2^e for |e| up to ~3000, as exact power-of-two products (barring over/underflow).
__device__ __forceinline__ double scale2(double v, int e)
{
    while (e > 1000) { v *= pow2i(1000); e -= 1000; }
    while (e < -1000) { v *= pow2i(-1000); e += 1000; }
    return v * pow2i(e);
}

// 1 / a by Smith's scaled formula (R. L. Smith, "Algorithm 116: Complex
// division", CACM 5(8), 1962): with |p| >= |q| the larger and smaller of
// |Re a|, |Im a|, r = q / p, d = p + q r, and 1/a = (1 - i r) / d or (r - i) / d.
__device__ __forceinline__ double2 c_rcp(double2 a)
{
    const bool re_big = abs_bits(a.x) >= abs_bits(a.y);
    const double pbig = re_big ? a.x : a.y;
    const double qsml = re_big ? a.y : a.x;
    const double r = qsml / pbig;
    const double d = fma(qsml, r, pbig);
    const double id = 1.0 / d;
    const double rid = r * id;
    return re_big ? make_double2(id, -rid) : make_double2(rid, -id);
}

// Rows of the warp block that the Lanczos sweeps ask L2 to fetch ahead of use. The
// one-row register prefetch of each sweep covers one row of the warp's own work,
// which in sweeps (a) and (e) is shorter than a round trip to HBM when a warp has
// its scheduler alone (the end of a launch). The bulk L2 prefetch kPfRows rows
// ahead, issued by one lane and holding no registers, turns those loads into L2
// hits: 12 % faster with one warp per scheduler, 1 % with two.
constexpr int kPfRows = 4;



// Asks L2 to fetch `bytes` bytes at `src` (16-byte aligned, a multiple of 16): one
// bulk-copy prefetch (no destination, no completion to wait for).
__device__ __forceinline__ void l2_prefetch(const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// SplitMix64 output number c for `seed` (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long c)
{
    unsigned long long z = seed + (c + 1ULL) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------- Ritz value
// Characteristic polynomial p_k(x) = det(xI - T_k) of the Lanczos tridiagonal
// (alpha_i = Ta[i*P], beta_i^2 = Tb[i*P]) and its derivative by the three-term
// recurrence, rescaled by powers of two; returns true when every p_i(x) > 0,
// i.e. x lies above every eigenvalue of T_k (Sturm).
__device__ __forceinline__ bool charpoly(const double *Ta, const double *Tb, int64_t P, int k, double x,
                                         double &pk, double &dpk)
{
    double p = x - Ta[0], pp = 1.0, dp = 1.0, dpp = 0.0;
    int neg = __double2hiint(p);  // sign bit collects any p_i <= 0 (zero checked below)
    bool zero = (p == 0.0);
    for (int i = 1; i < k; ++i) {
        const double a = Ta[(int64_t)i * P];
        const double b2 = Tb[(int64_t)(i - 1) * P];
        const double tt = x - a;
        const double pn = fma(tt, p, -(b2 * pp));
        const double dpn = fma(tt, dp, fma(-b2, dpp, p));
        pp = p; p = pn; dpp = dp; dp = dpn;
        neg |= __double2hiint(p);
        zero |= (__double_as_longlong(p) << 1) == 0;
        const int e = exp_field(p);
        if (e > 1023 + 480 || (e < 1023 - 480 && e != 0)) {
            const double s = pow2i(1023 - e);
            p *= s; pp *= s; dp *= s; dpp *= s;
        }
    }
    pk = p;
    dpk = dp;
    return neg >= 0 && !zero;
}

// Largest eigenvalue of T_k from the Gershgorin upper bound (no previous Ritz
// value known): Newton from above, lower bound max_i alpha_i.
__device__ __forceinline__ double ritz_top_cold(const double *Ta, const double *Tb, int64_t P, int k)
{
    double hi = -1.7e308, lo = -1.7e308, bprev = 0.0;
    for (int i = 0; i < k; ++i) {
        const double a = Ta[(int64_t)i * P];
        const double b = (i < k - 1) ? sqrt(Tb[(int64_t)i * P]) : 0.0;
        hi = fmax(hi, a + bprev + b);
        lo = fmax(lo, a);
        bprev = b;
    }
    double pk, dpk, x = hi;
    (void)charpoly(Ta, Tb, P, k, x, pk, dpk);
    for (int it = 0; it < 200; ++it) {
        const double d = pk / dpk;
        double xn = x - d;
        if (!(xn >= lo)) xn = lo;
        const bool done = !(fabs(d) > fabs(x) * 0x1.0p-51) || xn == x;
        x = xn;
        if (done) break;
        (void)charpoly(Ta, Tb, P, k, x, pk, dpk);
    }
    return x;
}

// Largest eigenvalue of T_k, k >= 2, given theta_prev = lambda_max(T_{k-1}),
// its last increment dprev, alpha_k and beta_{k-1}^2. Newton from above on
// p_k is monotone; the start is the first of a few trial points above
// theta_prev that the Sturm test accepts, else the Weyl bound
// max(theta_prev, alpha_k) + beta_{k-1}.
__device__ __forceinline__ double ritz_top(const double *Ta, const double *Tb, int64_t P, int k,
                                           double theta_prev, double dprev, double alpha_k, double b2)
{
    double pk, dpk;
    double x = 0.0;
    bool ok = false;
    double step = fmax(2.0 * dprev, fabs(theta_prev) * 0x1.0p-40);
    for (int m = 0; m < 4 && !ok; ++m) {
        x = theta_prev + step;
        ok = charpoly(Ta, Tb, P, k, x, pk, dpk);
        step *= 16.0;
    }
    if (!ok) {
        x = fmax(theta_prev, alpha_k) + sqrt(b2);
        (void)charpoly(Ta, Tb, P, k, x, pk, dpk);
    }
    for (int it = 0; it < 64; ++it) {
        const double d = pk / dpk;
        double xn = x - d;
        if (!(xn >= theta_prev)) xn = theta_prev;  // interlacing: theta_k >= theta_{k-1}
        const bool done = !(fabs(d) > x * 0x1.0p-51) || xn == x;
        x = xn;
        if (done) break;
        (void)charpoly(Ta, Tb, P, k, x, pk, dpk);
    }
    return x;
}

// ------------------------------------------------------------------ kernel
// Per-warp workspace block (one block per warp, the warp's 32 lanes interleaved
// in 16-byte units so that every access of a warp is 512 contiguous bytes):
//   row record j (row_bytes apart):  field f at f * 512 for f = 0 .. S+2
//       f = 0            1 / U_jj
//       f = 1 .. KW      U_{j, j+f}
//       f = KW+1 .. S-1  multipliers l_{j+r, j}, r = 1 .. KL
//       f = S, S+1, S+2  Lanczos vectors Va (q), Vb (u / w), Vx (solve work)
//     then 32 pivot offsets (bytes)
//   after n rows: alpha_k [k_max][32] and beta_k^2 [k_max][32] doubles.
template <int KL, int KU>
struct Shape {
    static constexpr int KW = KL + KU;         // superdiagonals of U after fill-in
    static constexpr int S = 2 * KL + KU + 1;  // factor values per row
    static constexpr int FA = S, FB = S + 1, FX = S + 2;
    static constexpr int FY = S + 3;  // gradient kernel only: the Ritz vector
    // 12 warps per SM while the elimination window is small, else 8
    // two resident blocks per SM (kBlocksPerSm): up to 255 registers per thread
    static constexpr int MIN_BLOCKS = kBlocksPerSm;
};

// The matrix and grid a group belongs to (the launch's one matrix, or one of a batch).
struct Mat {
    const double2 *bands;
    const double2 *q1;
    int n, nx, ny;
    double re_min, im_min, hx, hy;
    int64_t out_off;
};

__device__ __forceinline__ Mat single_mat(const KParams &p)
{
    return Mat{p.bands, p.q1, p.n, p.nx, p.ny, p.re_min, p.im_min, p.hx, p.hy, 0};
}

__device__ __forceinline__ Mat plan_mat(const KParams &p, int m)
{
    const PlanMat &e = p.pmats[m];
    return Mat{e.bands, p.q1 + e.q1_off, e.n, e.nx, e.ny, e.re_min, e.im_min, e.hx, e.hy, e.out_off};
}

// Batch: the matrix whose group range holds global group g (binary search on gstart).
__device__ __forceinline__ int plan_find(const KParams &p, int64_t g)
{
    int lo = 0, hi = p.nmats - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.pmats[mid].gstart <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Batch: the matrix whose estimate-chunk range holds chunk c.
__device__ __forceinline__ int plan_find_chunk(const KParams &p, int64_t c)
{
    int lo = 0, hi = p.nmats - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.pmats[mid].estart <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Lanczos scalars carried from step to step (see the kernel's header comment).
struct LzState {
    double acoef = 0.0;    // v_k = w_{k-1} - acoef v_{k-1}
    double beta_p = 0.0;   // beta_{k-1}
    double beta_pp = 0.0;  // beta_{k-2}
    int e1 = 0;            // binary exponent of the largest component of B^{-1} q_1
};

// One Lanczos step k on the point held by this lane: sweeps (a), (b), (d), (e).
// Returns -1 to go on, or the point's final status when the step ends the process
// (0: beta_{k-1} = 0, the Krylov space is exhausted and theta_{k-1} is exact; 5: a
// value left the double range). On return `alpha` holds alpha_k, beta_{k-1}^2 is in
// Tb and alpha_k in Ta. With ACC, sweep (a) also adds yc * v_k into the field FY (the
// Ritz vector of the gradient kernel); with only_a the step stops after sweep (a).
template <int KL, int KU, bool ACC>
__device__ __forceinline__ int lanczos_step(const KParams &p, const Mat &M, char *const rows, uint8_t *const pivs,
                                            double *const Ta, double *const Tb, const int k, LzState &st, double &alpha,
                                            const double yc, const bool only_a)
{
    using SH = Shape<KL, KU>;
    constexpr int KW = SH::KW;
    constexpr int FA = SH::FA, FB = SH::FB, FX = SH::FX;
    constexpr int64_t TS = 32;
    const int n = M.n;
    const int RB = p.row_bytes;
#define FLD(j, f) (*reinterpret_cast<double2 *>(rows + (j) * RB + (f) * 512))
#define PIVOF(j) (pivs[(j) * RB])
    // Rows of a sweep unrolled together, so that the scheduler can interleave the
    // independent products of consecutive rows (one warp per scheduler then keeps the
    // FP64 unit 71 % busy instead of 62 %); shapes whose elimination window or Ritz
    // vector field would spill registers keep one row.
    constexpr int kSweepUnroll = (!ACC && (KL + 1) * (KW + 1) <= 24) ? 2 : 1;
    const bool first = (k == 1);
    // L2 prefetch ranges of a row record (see kPfRows): the multipliers, v_k and
    // v_{k-1} [(KW+1) .. S+1] (+ the work field for sweep (e)), the pivot bytes, the
    // U fields [0 .. KW] and the work field FX
    char *const wb = rows - (threadIdx.x & 31) * 16;
    const bool pf_lane = kPfRows > 0 && (threadIdx.x & 31) == 0;
    constexpr unsigned kLBytes = (unsigned)(KL + 2) * 512u, kUBytes = (unsigned)(KW + 1) * 512u;
    auto pf_lvec = [&](int j, bool with_fx) {
        l2_prefetch(wb + (int64_t)j * RB + (KW + 1) * 512, with_fx ? kLBytes + 512u : kLBytes);
        if (KL > 0) l2_prefetch(wb + (int64_t)j * RB + p.piv_offset, 32u);
        if (ACC && !with_fx) l2_prefetch(wb + (int64_t)j * RB + SH::FY * 512, 512u);  // Ritz vector, sweep (a)
    };
    auto pf_u = [&](int j) {
        l2_prefetch(wb + (int64_t)j * RB, kUBytes);
        l2_prefetch(wb + (int64_t)j * RB + FX * 512, 512u);
    };
    const int fcur = (k & 1) ? FA : FB;   // v_k and, after (e), ...
    const int fprv = (k & 1) ? FB : FA;   // v_{k-1}, replaced by w_k in (e)
    // (a) v_k = w_{k-1} - st.acoef v_{k-1} (q_1 at k = 1); |v_k|^2; interchanges + L forward
    double b2 = 0.0;
    {
        double2 X[KL + 1];
        // y: the Ritz vector's current value at row ii (ACC only), loaded with the row's
        // other operands one row ahead
        auto make_v = [&](int ii, double2 w, double2 vp, double2 y) -> double2 {
            const double2 v = first ? w : make_double2(fma(-st.acoef, vp.x, w.x), fma(-st.acoef, vp.y, w.y));
            b2 = fma(v.x, v.x, fma(v.y, v.y, b2));
            FLD(ii, fcur) = v;
            if (ACC) FLD(ii, SH::FY) = make_double2(fma(yc, v.x, y.x), fma(yc, v.y, y.y));  // y += yc v_k
            return v;
        };
        auto load_w = [&](int ii, double2 &w, double2 &vp, double2 &y) {
            if (first) { w = __ldg(&M.q1[ii]); vp = make_double2(0.0, 0.0); }
            else { w = FLD(ii, fcur); vp = FLD(ii, fprv); }
            y = (ACC && !first) ? FLD(ii, SH::FY) : make_double2(0.0, 0.0);
        };
#pragma unroll
        for (int r = 0; r < KL; ++r) {
            X[r] = make_double2(0.0, 0.0);
            if (r < n) { double2 w, vp, y; load_w(r, w, vp, y); X[r] = make_v(r, w, vp, y); }
        }
        // row j needs pivot j, multipliers of column j and v_{j+KL}; prefetch row j+1
        double2 nl[KL + 1], nw = make_double2(0.0, 0.0), nvp = make_double2(0.0, 0.0), nyr = make_double2(0.0, 0.0);
        int npv = 0;
        auto load_a = [&](int j) {
            if (KL > 0) {
                npv = PIVOF(j);
#pragma unroll
                for (int r = 1; r <= KL; ++r) nl[r] = FLD(j, KW + r);
            }
            if (j + KL < n) load_w(j + KL, nw, nvp, nyr);
        };
        if (pf_lane)
            for (int j = 0; j < kPfRows && j < n; ++j) pf_lvec(j, false);
        load_a(0);
#pragma unroll kSweepUnroll
        for (int j = 0; j < n; ++j) {
            if (pf_lane && j + kPfRows < n) pf_lvec(j + kPfRows, false);
            double2 cl[KL + 1];
#pragma unroll
            for (int r = 1; r <= KL; ++r) cl[r] = nl[r];
            const int cpv = npv;
            const double2 cw = nw, cvp = nvp, cy = nyr;
            if (j + 1 < n) load_a(j + 1);
            X[KL] = (j + KL < n) ? make_v(j + KL, cw, cvp, cy) : make_double2(0.0, 0.0);
            if (KL > 0) {
#pragma unroll
                for (int r = 1; r <= KL; ++r) {
                    const bool s = (cpv == r);
                    const double2 a = X[0], b = X[r];
                    X[0] = s ? b : a;
                    X[r] = s ? a : b;
                }
#pragma unroll
                for (int r = 1; r <= KL; ++r) X[r] = c_sub_mul(X[r], cl[r], X[0]);
            }
            FLD(j, FX) = X[0];
#pragma unroll
            for (int r = 0; r < KL; ++r) X[r] = X[r + 1];
        }
    }
    if (only_a) return -1;
    double invb = 1.0;
    if (!first) {
        if (b2 == 0.0) return 0;  // Krylov space exhausted: theta_{k-1} exact
        if (!(b2 <= 1.7e308)) return 5;  // overflow: sigma below range
        Tb[(int64_t)(k - 2) * TS] = b2;  // beta_{k-1}^2 = |v_k|^2 completes T_{k-1}
        st.beta_pp = st.beta_p;
        st.beta_p = sqrt(b2);
        invb = 1.0 / st.beta_p;
    }

    // (b) U x = Vx backward; x_j = (Vx_j - sum U_{j,j+c} x_{j+c}) / U_jj
    int emax = 0;
    {
        double2 Y[KW + 1];
#pragma unroll
        for (int c = 0; c <= KW; ++c) Y[c] = make_double2(0.0, 0.0);
        double2 nu[KW + 1], nv;
        auto load_b = [&](int j) {
#pragma unroll
            for (int c = 0; c <= KW; ++c) nu[c] = FLD(j, c);
            nv = FLD(j, FX);
        };
        if (pf_lane)
            for (int j = n - 1; j >= n - kPfRows && j >= 0; --j) pf_u(j);
        load_b(n - 1);
#pragma unroll kSweepUnroll
        for (int j = n - 1; j >= 0; --j) {
            if (pf_lane && j - kPfRows >= 0) pf_u(j - kPfRows);
            double2 cu[KW + 1];
#pragma unroll
            for (int c = 0; c <= KW; ++c) cu[c] = nu[c];
            double2 acc = nv;
            if (j > 0) load_b(j - 1);
#pragma unroll
            // oldest x first: only the last term waits for x_{j+1}, so the chain of row
            // j overlaps the end of row j+1 (the loop is unrolled by kSweepUnroll)
            for (int c = KW; c >= 1; --c) acc = c_sub_mul(acc, cu[c], Y[c]);
            const double2 x = c_mul(acc, cu[0]);
            emax = max(emax, max(exp_field(x.x), exp_field(x.y)));
            FLD(j, FX) = x;
#pragma unroll
            for (int c = KW; c >= 2; --c) Y[c] = Y[c - 1];
            if (KW >= 1) Y[1] = x;
        }
    }
    if (emax >= 2047) return 5;
    // x is rescaled by 2^-es at the first step (fixing st.e1), at every step of
    // a point with |st.e1| > 450, and at any step whose y (about x 2^st.e1) could
    // come near the top of the double range. The decision is taken per warp;
    // an exact power-of-two scale leaves every lane's result unchanged.
    const bool scaled = __any_sync(__activemask(), first || st.e1 > 450 || st.e1 < -450 ||
                                                       (emax - 1023) + st.e1 + 24 > 1000);
    const int es = scaled ? clampi(emax - 1023, -1000, 1000) : 0;
    if (first) st.e1 = es;
    const double sc = pow2i(-es);

    // (d) U^* t = x * 2^-es forward, accumulators for rows i..i+KW
    {
        double2 Acc[KW + 1];
#pragma unroll
        for (int c = 0; c < KW; ++c) {
            double2 v = make_double2(0.0, 0.0);
            if (c < n) { v = FLD(c, FX); if (scaled) { v.x *= sc; v.y *= sc; } }
            Acc[c] = v;
        }
        double2 nu[KW + 1], nv = make_double2(0.0, 0.0);
        auto load_d = [&](int i) {
#pragma unroll
            for (int c = 0; c <= KW; ++c) nu[c] = FLD(i, c);
            nv = (i + KW < n) ? FLD(i + KW, FX) : make_double2(0.0, 0.0);
        };
        if (pf_lane)
            for (int i = 0; i < kPfRows && i < n; ++i) pf_u(i);
        load_d(0);
#pragma unroll kSweepUnroll
        for (int i = 0; i < n; ++i) {
            if (pf_lane && i + kPfRows < n) pf_u(i + kPfRows);
            double2 cu[KW + 1];
#pragma unroll
            for (int c = 0; c <= KW; ++c) cu[c] = nu[c];
            Acc[KW] = scaled ? make_double2(nv.x * sc, nv.y * sc) : nv;
            if (i + 1 < n) load_d(i + 1);
            const double2 tt = c_mul_conj(Acc[0], cu[0]);
            FLD(i, FX) = tt;
#pragma unroll
            for (int c = 1; c <= KW; ++c) Acc[c] = c_sub_conjmul(Acc[c], cu[c], tt);
#pragma unroll
            for (int c = 0; c < KW; ++c) Acc[c] = Acc[c + 1];
        }
    }

    // (e) L^* backward with interchanges; as each y_i becomes final,
    //     w_i = F y_i - G v_{k-1,i} (= (H' q_k - beta_{k-1} q_{k-1})_i)
    //     and asum += Re(conj(v_{k,i}) w_i)
    const double F = scale2(first ? 1.0 : invb, es - 2 * st.e1);
    const double G = (k == 2) ? st.beta_p : st.beta_p / (st.beta_pp > 0.0 ? st.beta_pp : 1.0);
    double asum = 0.0;
    {
        auto emit = [&](int ii, double2 y, double2 vc, double2 vp) {
            const double2 w = first ? make_double2(F * y.x, F * y.y)
                                    : make_double2(fma(F, y.x, -(G * vp.x)), fma(F, y.y, -(G * vp.y)));
            asum = fma(vc.x, w.x, fma(vc.y, w.y, asum));
            FLD(ii, fprv) = w;
        };
        double2 T[KL + 1];
#pragma unroll
        for (int r = 0; r <= KL; ++r) T[r] = make_double2(0.0, 0.0);
        // row j needs t_j, multipliers of column j, pivot j and v_k, v_{k-1} at j + KL
        double2 nl[KL + 1], nt, nvc = make_double2(0.0, 0.0), nvp = make_double2(0.0, 0.0);
        int npv = 0;
        auto load_e = [&](int j) {
            nt = FLD(j, FX);
            if (KL > 0) {
                npv = PIVOF(j);
#pragma unroll
                for (int r = 1; r <= KL; ++r) nl[r] = FLD(j, KW + r);
            }
            if (j + KL < n) {
                nvc = FLD(j + KL, fcur);
                nvp = first ? make_double2(0.0, 0.0) : FLD(j + KL, fprv);
            }
        };
        if (pf_lane)
            for (int j = n - 1; j >= n - kPfRows && j >= 0; --j) pf_lvec(j, true);
        load_e(n - 1);
#pragma unroll kSweepUnroll
        for (int j = n - 1; j >= 0; --j) {
            if (pf_lane && j - kPfRows >= 0) pf_lvec(j - kPfRows, true);
            double2 cl[KL + 1];
#pragma unroll
            for (int r = 1; r <= KL; ++r) cl[r] = nl[r];
            const int cpv = npv;
            const double2 ct = nt, cvc = nvc, cvp = nvp;
            if (j > 0) load_e(j - 1);
#pragma unroll
            for (int r = KL; r >= 1; --r) T[r] = T[r - 1];
            T[0] = ct;
            if (KL > 0) {
#pragma unroll
                for (int r = KL; r >= 1; --r) T[0] = c_sub_conjmul(T[0], cl[r], T[r]);  // oldest first
#pragma unroll
                for (int r = 1; r <= KL; ++r) {
                    const bool s = (cpv == r);
                    const double2 a = T[0], b = T[r];
                    T[0] = s ? b : a;
                    T[r] = s ? a : b;
                }
                if (j + KL < n) emit(j + KL, T[KL], cvc, cvp);
            } else {
                emit(j, T[0], cvc, cvp);
            }
        }
#pragma unroll
        for (int r = 0; r < KL; ++r)
            if (r < n) emit(r, T[r], FLD(r, fcur), first ? make_double2(0.0, 0.0) : FLD(r, fprv));
    }
    // alpha_k = Re<q_k, w_k> = asum / beta_{k-1} (asum at k = 1, v_1 = q_1);
    // v_{k+1} = w_k - alpha_k q_k = w_k - (alpha_k / beta_{k-1}) v_k
    alpha = first ? asum : asum * invb;
    st.acoef = first ? alpha : alpha * invb;
    Ta[(int64_t)(k - 1) * TS] = alpha;
    return -1;
#undef FLD
#undef PIVOF
}

// Banded LU of B = zI - A with partial pivoting inside the band, for the point z
// held by this lane (all 32 lanes of the warp call it together; lanes without a
// point pass a dummy z). A's diagonals for rows R0 .. R0+31 are staged in this
// warp's shared-memory window Aw with one coalesced 512-byte load per diagonal:
//   Aw[c][r - R0] = A[r][r + c - KL] = bands[c * n + r],  c = 0 .. KW.
// The pivot of column j is the row of largest |Re| + |Im| among rows j .. j+KL (the
// first on ties); U gains KL superdiagonals; the row record j keeps 1/U_jj, the
// KW superdiagonal entries of U and the KL multipliers. Returns true when a column
// had no nonzero pivot candidate (B singular).
template <int KL, int KU>
__device__ __forceinline__ bool band_lu(const KParams &p, const Mat &M, char *const rows, uint8_t *const pivs,
                                        double2 (*const Aw)[32], const int lane, const double zr, const double zi,
                                        const bool bad_input)
{
    using SH = Shape<KL, KU>;
    constexpr int KW = SH::KW;
    const int n = M.n;
    const int RB = p.row_bytes;
#define FLD(j, f) (*reinterpret_cast<double2 *>(rows + (j) * RB + (f) * 512))
#define PIVOF(j) (pivs[(j) * RB])
int R0 = 0;
auto stage = [&](int r0) {
    __syncwarp();
#pragma unroll
    for (int c = 0; c <= KW; ++c) {
        const int r = r0 + lane;
        Aw[c][lane] = (r < n) ? __ldg(&M.bands[(int64_t)c * n + r]) : make_double2(0.0, 0.0);
    }
    __syncwarp();
};
if (!bad_input) stage(0);
double2 W[KL + 1][KW + 1];
#pragma unroll
for (int r = 0; r <= KL; ++r)
#pragma unroll
    for (int c = 0; c <= KW; ++c) {
        const int d = c - r;
        double2 v = make_double2(0.0, 0.0);
        if (!bad_input && d >= -KL && d <= KU && r < n && c < n) {
            const double2 a = Aw[d + KL][r];
            v = (d == 0) ? make_double2(zr - a.x, zi - a.y) : make_double2(-a.x, -a.y);
        }
        W[r][c] = v;
    }
bool singular = false;
for (int j = 0; j < (bad_input ? 0 : n); ++j) {
    int pr = 0;
    unsigned long long best = abs_bits(fabs(W[0][0].x) + fabs(W[0][0].y));
#pragma unroll
    for (int r = 1; r <= KL; ++r) {
        const unsigned long long v = abs_bits(fabs(W[r][0].x) + fabs(W[r][0].y));
        if (v > best) { best = v; pr = r; }
    }
#pragma unroll
    for (int r = 1; r <= KL; ++r) {
        const bool s = (pr == r);
#pragma unroll
        for (int c = 0; c <= KW; ++c) {
            const double2 a = W[0][c], b = W[r][c];
            W[0][c] = s ? b : a;
            W[r][c] = s ? a : b;
        }
    }
    // an exact zero pivot column: B is singular; the lane keeps stepping with a
    // unit pivot (its factor is not used) so that the warp stays together
    if (best == 0ULL) { singular = true; W[0][0] = make_double2(1.0, 0.0); }
    const double2 rp = c_rcp(W[0][0]);
    FLD(j, 0) = rp;
#pragma unroll
    for (int c = 1; c <= KW; ++c) FLD(j, c) = W[0][c];
    if (KL > 0) PIVOF(j) = (uint8_t)pr;
#pragma unroll
    for (int r = 1; r <= KL; ++r) {
        const double2 l = c_mul(W[r][0], rp);
        FLD(j, KW + r) = l;
#pragma unroll
        for (int c = 1; c <= KW; ++c) W[r][c] = c_sub_mul(W[r][c], l, W[0][c]);
    }
#pragma unroll
    for (int r = 0; r < KL; ++r) {
#pragma unroll
        for (int c = 0; c < KW; ++c) W[r][c] = W[r + 1][c + 1];
        W[r][KW] = make_double2(0.0, 0.0);
    }
    const int i = j + 1 + KL;  // next row, columns j+1 .. j+1+KW (d = c - KL)
    if (i - R0 >= 32) { R0 += 32; stage(R0); }
#pragma unroll
    for (int c = 0; c <= KW; ++c) {
        const int col = j + 1 + c;
        double2 v = make_double2(0.0, 0.0);
        if (i < n && col < n) {
            const double2 a = Aw[c][i - R0];
            v = (c == KL) ? make_double2(zr - a.x, zi - a.y) : make_double2(-a.x, -a.y);
        }
        W[KL][c] = v;
    }
}

    return singular;
#undef FLD
#undef PIVOF
}

// The Lanczos process of one point (the lane's), advanced one step at a time.
struct LzRun {
    LzState st;
    double theta = 0.0, theta_prev = 0.0, dprev = 0.0;
    int k = 0;       // steps taken
    int kth = 0;     // step whose Ritz value `theta` holds
    int ksteps = 0;  // steps that produced a Ritz value
};

// Step k + 1 of the Lanczos process on H' = (B B^*)^{-1} / 2^(2 e1) after band_lu, with
// the Ritz value and the stopping test. Returns -1 to go on, else the point's status:
// 0 converged (or beta = 0: the Krylov space is exhausted), 2 k_max reached without
// meeting the test, 5 a value left the double range.
template <int KL, int KU>
__device__ __forceinline__ int lz_advance(const KParams &p, const Mat &M, char *const rows, uint8_t *const pivs,
                                          double *const Ta, double *const Tb, LzRun &r)
{
    constexpr int64_t TS = 32;
    // The stored Lanczos vectors are v_k = u_k = beta_{k-1} q_k (v_1 = q_1), not
    // normalised: 1/beta rides on the scalars of the next sweep. 2^e1 is the
    // binary exponent of the largest component of B^{-1} q_1 (about 1/sigma);
    // for |e1| <= 450 the solves of later steps stay inside the double range
    // (x ~ beta 2^e1, y ~ beta 2^(2 e1) theta') and need no rescaling.
    const int kmax = p.k_max;
    const int kr0 = max(1, min(p.k_min, kmax) - 1);  // first step whose Ritz value is needed
    const int kc0 = max(2, p.k_min);                 // first step with a stopping test
    const int k = r.k + 1;
    double alpha = 0.0;
    const int rs = lanczos_step<KL, KU, false>(p, M, rows, pivs, Ta, Tb, k, r.st, alpha, 0.0, false);
    r.k = k;
    if (rs >= 0) return rs;
    r.ksteps = k;
    if (k >= kr0) {
        double th;
        if (k == 1) th = alpha;
        else if (r.kth == k - 1) th = ritz_top(Ta, Tb, TS, k, r.theta, r.dprev, alpha, r.st.beta_p * r.st.beta_p);
        else th = ritz_top_cold(Ta, Tb, TS, k);
        const bool have_prev = (r.kth == k - 1);
        r.theta_prev = r.theta;
        r.theta = th;
        r.kth = k;
        r.dprev = have_prev ? r.theta - r.theta_prev : 0.0;
        if (k >= kc0 && have_prev && r.theta - r.theta_prev <= p.tol * r.theta) return 0;
    }
    return k >= kmax ? 2 : -1;
}

// sigma = 2^(-e1) / sqrt(theta) from the final Ritz value (recomputed when the last
// step's was skipped); UNDERFLOW (5, sigma = 0) when theta left the double range.
template <int KL, int KU>
__device__ __forceinline__ int lz_finish(double *const Ta, double *const Tb, LzRun &r, int status, double &sigma)
{
    constexpr int64_t TS = 32;
    sigma = 0.0;
    if (status != 5 && r.kth != r.ksteps && r.ksteps >= 1) {
        r.theta = (r.ksteps == 1) ? Ta[0] : ritz_top_cold(Ta, Tb, TS, r.ksteps);
        r.kth = r.ksteps;
    }
    if (status != 5) {
        if (!(r.theta > 0.0) || !(r.theta <= 1.7e308)) status = 5;
        else sigma = (1.0 / sqrt(r.theta)) * pow2i(clampi(-r.st.e1, -1022, 1023));
    }
    if (status == 5) sigma = 0.0;
    return status;
}

// Lanczos on H' for the point held by this lane, after band_lu: steps until the
// stopping test, beta = 0 or k_max. Returns the point's status (0 OK, 2
// NOT_CONVERGED, 5 UNDERFLOW) and sets sigma, the steps taken, the final Ritz value
// theta (in H' units) and the Lanczos scalars st.
template <int KL, int KU>
__device__ __forceinline__ int lanczos_sigma(const KParams &p, const Mat &M, char *const rows, uint8_t *const pivs,
                                             double *const Ta, double *const Tb, LzState &st, double &sigma, int &ksteps,
                                             double &theta)
{
    LzRun r;
    int status;
    while ((status = lz_advance<KL, KU>(p, M, rows, pivs, Ta, Tb, r)) < 0) {
    }
    status = lz_finish<KL, KU>(Ta, Tb, r, status, sigma);
    st = r.st;
    ksteps = r.ksteps;
    theta = r.theta;
    return status;
}

// Flat grid index of lane `lane` of group g (-1: no point): on the full grid an
// 8 x 4 tile (8 abscissae, 4 ordinates) of M's grid (g counted within M), whose
// neighbouring points take similar Lanczos step counts so the warp's lanes stay
// busy together; in restricted mode 32 consecutive entries of the list.
__device__ __forceinline__ int64_t group_point(const KParams &p, const Mat &M, int64_t g, int lane)
{
    const int64_t ngrid = (int64_t)M.nx * M.ny;
    if (p.idx) {
        const int64_t pt = g * 32 + lane;
        if (pt >= p.npts) return -1;
        const int64_t f = (int64_t)p.idx[pt];
        return (f >= 0 && f < ngrid) ? f : -1;
    }
    const int tiles_x = (M.nx + 7) >> 3;
    const int ty = (int)(g / tiles_x), tx = (int)(g - (int64_t)ty * tiles_x);
    const int i = ty * 4 + (lane >> 3), j = tx * 8 + (lane & 7);
    return (i < M.ny && j < M.nx) ? (int64_t)i * M.nx + j : -1;
}

// A point representative of group g for the work-order estimate: the tile's point
// (1, 3) (clamped to the grid), or the first entry of a list chunk.
__device__ __forceinline__ int64_t group_anchor(const KParams &p, const Mat &M, int64_t g)
{
    const int64_t ngrid = (int64_t)M.nx * M.ny;
    if (p.idx) {
        const int64_t f = (int64_t)p.idx[g * 32];
        return (f >= 0 && f < ngrid) ? f : -1;
    }
    const int tiles_x = (M.nx + 7) >> 3;
    const int ty = (int)(g / tiles_x), tx = (int)(g - (int64_t)ty * tiles_x);
    const int i = min(ty * 4 + 1, M.ny - 1), j = min(tx * 8 + 3, M.nx - 1);
    return (int64_t)i * M.nx + j;
}

// Outputs of one point: sigma, the eps-mask bits, status and steps.
__device__ __forceinline__ void write_point(const KParams &p, int64_t flat, double sigma, int status, int ksteps)
{
    p.sigma[flat] = sigma;
    if (p.mask) {
        uint32_t bits = 0;
        const unsigned long long sb = abs_bits(sigma);
        for (int l = 0; l < p.n_eps; ++l) bits |= (sb <= abs_bits(p.eps[l]) ? 1u : 0u) << l;
        p.mask[flat] = bits;
    }
    if (p.status) p.status[flat] = (int8_t)status;
    if (p.steps) p.steps[flat] = ksteps;
}

template <int KL, int KU>
__global__ void __launch_bounds__(kThreads, Shape<KL, KU>::MIN_BLOCKS) k_sigma_min(const KParams p)
{
    using SH = Shape<KL, KU>;
    constexpr int KW = SH::KW;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int RB = p.row_bytes;
    char *const wbase = p.wdata + warp * p.warp_bytes;
    char *const rows = wbase + lane * 16;
    uint8_t *const pivs = reinterpret_cast<uint8_t *>(wbase) + p.piv_offset + lane;
    double *const Ta = reinterpret_cast<double *>(wbase + (int64_t)p.trow * RB) + lane;
    double *const Tb = Ta + (int64_t)p.k_max * 32;
    __shared__ double2 Aw_all[kThreads / 32][KW + 1][32];
    double2 (*const Aw)[32] = Aw_all[threadIdx.x >> 5];
    double zr = 0.0, zi = 0.0;

#define FLD(j, f) (*reinterpret_cast<double2 *>(rows + (j) * RB + (f) * 512))
#define PIVOF(j) (pivs[(j) * RB])

    for (;;) {
        // the warp takes the next group of 32 points (estimate pass: 32 groups' anchors)
        int grp = 0;
        if (lane == 0) grp = atomicAdd(p.counter, 1);
        grp = __shfl_sync(0xffffffffu, grp, 0);
        if ((int64_t)grp >= (p.estimate ? p.nchunks : p.ngroups)) break;
        int64_t flat = -1;
        int64_t anchor_of = -1;  // estimate pass: the group whose anchor this lane runs
        Mat M;
        bool bad_input;
        if (p.estimate) {
            // the lanes of one warp run the anchors of 32 groups of one matrix
            int64_t a = (int64_t)grp * 32 + lane, g0 = 0, gn = p.ngroups;
            if (p.nmats) {
                const int m = plan_find_chunk(p, grp);
                M = plan_mat(p, m);
                bad_input = p.mflags[m] != 0;
                a = (grp - p.pmats[m].estart) * 32 + lane;
                g0 = p.pmats[m].gstart;
                gn = (int64_t)((M.nx + 7) / 8) * ((M.ny + 3) / 4);
            } else {
                M = single_mat(p);
                bad_input = p.flags[0] != 0;
            }
            if (a < gn) {
                anchor_of = g0 + a;
                flat = group_anchor(p, M, a);
            }
        } else {
            const int64_t g = p.order ? (int64_t)p.order[grp] : (int64_t)grp;
            int64_t gl = g;
            if (p.nmats) {
                const int m = plan_find(p, g);
                M = plan_mat(p, m);
                bad_input = p.mflags[m] != 0;
                gl = g - p.pmats[m].gstart;
            } else {
                M = single_mat(p);
                bad_input = p.flags[0] != 0;
            }
            flat = group_point(p, M, gl, lane);
        }
        // every lane runs the factorisation (lanes without a point on a dummy z), so
        // that the warp can stage the bands of A cooperatively
        const bool have = flat >= 0;
        if (p.estimate && anchor_of >= 0 && !have) {  // no valid anchor: file the group first-to-last
            p.sched_bucket[anchor_of] = 0;
            atomicAdd(&p.sched_hist[0], 1);
        }
        {
            const int gi = have ? (int)(flat / M.nx) : 0;
            const int gj = have ? (int)(flat - (int64_t)gi * M.nx) : 0;
            zr = fma((double)gj, M.hx, M.re_min);
            zi = fma((double)gi, M.hy, M.im_min);
        }

        // ---------------- 1. banded LU with partial pivoting
        const bool singular = band_lu<KL, KU>(p, M, rows, pivs, Aw, lane, zr, zi, bad_input);

        if (have) {
            double sigma = 0.0;
            int status = bad_input ? 3 : 1;  // NONFINITE input, else SINGULAR
            int ksteps = 0;
            if (!singular && !bad_input) {
                LzState st;
                double theta = 0.0;
                status = lanczos_sigma<KL, KU>(p, M, rows, pivs, Ta, Tb, st, sigma, ksteps, theta);
            }

            // ---------------- 4. outputs
            if (p.estimate) {
                // file the group under its estimated cost: the matrix order n (two buckets
                // per octave) and then sigma relative to the grid's extent (8 buckets per
                // octave over [2^-8, 1]): points far from the spectrum take the most
                // Lanczos steps. Groups are later taken in decreasing bucket order.
                int b = 0;
                if ((status == 0 || status == 2) && sigma > 0.0) {
                    const double ext = fmax(M.hx * (double)(M.nx - 1), M.hy * (double)(M.ny - 1));
                    const double rel = ext > 0.0 ? sigma / ext : sigma;
                    const int sb = clampi(8 * (exp_field(rel) - 1023) + ((__double2hiint(rel) >> 17) & 7) + 64, 1, 63);
                    const int nb = clampi(2 * (exp_field((double)M.n) - 1023) + ((__double2hiint((double)M.n) >> 19) & 1), 0,
                                          kBuckets / 64 - 1);
                    b = nb * 64 + sb;
                }
                p.sched_bucket[anchor_of] = b;
                atomicAdd(&p.sched_hist[b], 1);
                continue;
            }
            write_point(p, flat + M.out_off, sigma, status, ksteps);
        }
    }
#undef FLD
#undef PIVOF
}

template <int KL, int KU>
cudaError_t launch_sigma_min(const KParams &p, cudaStream_t stream)
{
    const int threads = (p.P % kThreads == 0) ? kThreads : 32;
    k_sigma_min<KL, KU><<<(unsigned)(p.P / threads), threads, 0, stream>>>(p);
    return cudaGetLastError();
}

template <int KL, int KU>
cudaError_t blocks_per_sm(int *nb)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_sigma_min<KL, KU>, kThreads, 0);
}

}  // namespace dev

// Launch and occupancy entry points for one kl and ku = 0 .. kMaxKU.
template <int KL>
KernelOps kernel_ops_for_ku(int ku)
{
    switch (ku) {
#define PSA_KU_CASE(K) case K: return KernelOps{&dev::launch_sigma_min<KL, K>, &dev::blocks_per_sm<KL, K>};
    PSA_KU_CASE(0) PSA_KU_CASE(1) PSA_KU_CASE(2) PSA_KU_CASE(3) PSA_KU_CASE(4)
    PSA_KU_CASE(5) PSA_KU_CASE(6) PSA_KU_CASE(7) PSA_KU_CASE(8)
#undef PSA_KU_CASE
    default: return KernelOps{nullptr, nullptr};
    }
}

}  // namespace psa
