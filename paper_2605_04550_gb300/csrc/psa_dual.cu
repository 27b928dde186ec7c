// psa_dual.cu -- the paper's dual-path classifier (Sec. 3.2.2): a coordinate
// pathway on the Fourier encoding phi(c) of the grid point (26 -> 64 -> 64), a
// matrix pathway on the per-point and global features f(z, A) (-> 128 -> 64),
// their concatenation h3 (128), a residual block h4 = SiLU(W4 h3 + b4),
// h5 = SiLU(W5 h4 + b5), h6 = h4 + h5, a projection h7 = SiLU(W7 h6 + b7) (64)
// and the sigmoid output p = sigma(w . h7 + b); SiLU throughout. Training is
// Adam on binary cross-entropy (Sec. 3.4), as for the MLP of psa_mlp.cu.
//
// The two pathways run as two fused GEMMs on the tensor cores: layer A maps the
// 128-wide feature row to [h_c1 (64) | h_m1 (128) | 64 zero columns] with a
// block-structured weight (coordinate rows read only the Fourier columns, matrix
// rows only the feature columns), and layer B maps that to [h_c2 (64) | h_m2 (64)]
// = h3 with a block-diagonal weight, so the concatenation costs nothing. The
// structural zeros are no parameters: their gradients are masked before Adam, so
// they stay zero and the fused network computes exactly the two separate
// pathways. The 64-wide projection is padded to the GEMM's 128 columns with zero
// rows (masked the same way). The residual sum h4 + h5 is added in the epilogue
// of layer 5's GEMM, and the backward pass adds dh6 to dh4 in the epilogue of the
// GEMM that forms W5^T dz5.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "psa.h"
#include "psa_gemm.h"

namespace psa {
namespace dual {

using mlp::GemmArgs;
using mlp::TILE;

constexpr int IN = PSA_MLP_IN;        // feature row width (psa_point_features)
constexpr int NC = 26;                // Fourier columns [0, 26)
constexpr int MC0 = 26, NMF = 35;     // matrix-path columns [26, 61)
constexpr int HC = 64, HM1 = 128, HM2 = 64, H3 = 128, H7 = 64;
constexpr int NA = 256;               // layer A outputs: [0, 64) coordinate, [64, 192) matrix, pad
constexpr int NB = 128, NH = 128;     // layer B outputs (= h3) and the residual block's width
static_assert(MC0 + NMF <= IN && HC + HM1 <= NA && HC + HM2 == H3, "layout");

// parameter vector (float32), padded matrices [out][in] row-major
constexpr int64_t OFF_WA = 0;
constexpr int64_t OFF_BA = OFF_WA + (int64_t)NA * IN;
constexpr int64_t OFF_WB = OFF_BA + NA;
constexpr int64_t OFF_BB = OFF_WB + (int64_t)NB * NA;
constexpr int64_t OFF_W4 = OFF_BB + NB;
constexpr int64_t OFF_B4 = OFF_W4 + (int64_t)NH * NH;
constexpr int64_t OFF_W5 = OFF_B4 + NH;
constexpr int64_t OFF_B5 = OFF_W5 + (int64_t)NH * NH;
constexpr int64_t OFF_W7 = OFF_B5 + NH;
constexpr int64_t OFF_B7 = OFF_W7 + (int64_t)NH * NH;
constexpr int64_t OFF_W8 = OFF_B7 + NH;
constexpr int64_t OFF_B8 = OFF_W8 + NH;
constexpr int64_t NPARAM = OFF_B8 + 1;
static_assert(NPARAM == PSA_DUAL_PARAMS, "parameter count");
constexpr int64_t FWD_CHUNK = 131072;

// Whether entry i of the parameter vector is a trainable parameter (else a
// structural zero of the fused layout).
__host__ __device__ inline bool is_param(int64_t i)
{
    if (i < OFF_BA) {
        const int r = (int)(i / IN), c = (int)(i % IN);
        return (r < HC && c < NC) || (r >= HC && r < HC + HM1 && c >= MC0 && c < MC0 + NMF);
    }
    if (i < OFF_WB) return i - OFF_BA < HC + HM1;
    if (i < OFF_BB) {
        const int r = (int)((i - OFF_WB) / NA), c = (int)((i - OFF_WB) % NA);
        return (r < HC && c < HC) || (r >= HC && c >= HC && c < HC + HM1);
    }
    if (i < OFF_W7) return true;  // bB, W4, b4, W5, b5
    if (i < OFF_B7) return (i - OFF_W7) / NH < H7;
    if (i < OFF_W8) return i - OFF_B7 < H7;
    if (i < OFF_B8) return i - OFF_W8 < H7;
    return i == OFF_B8;
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + __expf(-z)); }

// BF16 copies of the weights and, for training, of the transposes the input-gradient
// GEMMs take as their B operand (WB^T [NA][NB], W4^T, W5^T, W7^T [NH][NH]).
__global__ void k_dshadow(const float *theta, __nv_bfloat16 *wa, __nv_bfloat16 *wb, __nv_bfloat16 *w4,
                          __nv_bfloat16 *w5, __nv_bfloat16 *w7, __nv_bfloat16 *wbt, __nv_bfloat16 *w4t,
                          __nv_bfloat16 *w5t, __nv_bfloat16 *w7t)
{
    const int64_t na = (int64_t)NA * IN, nb = (int64_t)NB * NA, nh = (int64_t)NH * NH;
    const int64_t total = na + nb + 3 * nh;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < na) {
            wa[i] = __float2bfloat16_rn(theta[OFF_WA + i]);
            continue;
        }
        if (i < na + nb) {
            const int64_t q = i - na;
            const __nv_bfloat16 v = __float2bfloat16_rn(theta[OFF_WB + q]);
            wb[q] = v;
            if (wbt) wbt[(q % NA) * NB + q / NA] = v;
            continue;
        }
        const int64_t q = (i - na - nb) % nh, layer = (i - na - nb) / nh;
        const int64_t off = layer == 0 ? OFF_W4 : (layer == 1 ? OFF_W5 : OFF_W7);
        __nv_bfloat16 *w = layer == 0 ? w4 : (layer == 1 ? w5 : w7);
        __nv_bfloat16 *wt = layer == 0 ? w4t : (layer == 1 ? w5t : w7t);
        const __nv_bfloat16 v = __float2bfloat16_rn(theta[off + q]);
        w[q] = v;
        if (wt) wt[(q % NH) * NH + q / NH] = v;
    }
}

// x^T ([IN][rows]) of a batch, for layer A's weight gradient.
__global__ void k_dtranspose(const __nv_bfloat16 *x, __nv_bfloat16 *xt, int rows)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) t[k][threadIdx.x] = x[(int64_t)(r0 + k) * IN + c0 + threadIdx.x];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) xt[(int64_t)(c0 + k) * rows + r0 + threadIdx.x] = t[threadIdx.x][k];
}

// logit = h7 . w8 + b8 (w8 is zero past H7), one warp per row of h7 [rows][NH].
__device__ __forceinline__ float head_logit(const __nv_bfloat16 *h7, const float *theta, int64_t row, int lane)
{
    const uint2 v = *reinterpret_cast<const uint2 *>(h7 + row * NH + lane * 4);
    const __nv_bfloat16 *hb = reinterpret_cast<const __nv_bfloat16 *>(&v);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) s = fmaf(__bfloat162float(hb[j]), theta[OFF_W8 + lane * 4 + j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s + theta[OFF_B8];
}

__global__ void k_dhead(const __nv_bfloat16 *h7, const float *theta, float *prob, int64_t rows)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const float l = head_logit(h7, theta, row, lane);
    if (lane == 0) prob[row] = sigm(l);
}

// Mean binary cross-entropy (added to *loss), dL/dlogit = (sigmoid - y) / rows, d b8.
__global__ void k_dhead_train(const __nv_bfloat16 *h7, const float *theta, const float *y, float *dlogit, float *grad,
                              float *loss, int rows)
{
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const float l = head_logit(h7, theta, row, lane);
    if (lane == 0) {
        const float t = y[row];
        const float bce = fmaxf(l, 0.f) - l * t + log1pf(__expf(-fabsf(l)));
        const float d = (sigm(l) - t) / (float)rows;
        dlogit[row] = d;
        atomicAdd(loss, bce / (float)rows);
        atomicAdd(&grad[OFF_B8], d);
    }
}

// Backward through a SiLU layer of width W on a 32 x 32 tile: dz = dh * silu'(z),
// dh = dH[m][j] (ldw = W) or, for the projection layer, dlogit[m] * w8[j]; writes dz
// (BF16, row-major and transposed [W][rows]), adds the bias gradient into
// grad[off_b + j] and, for the projection layer, d w8[j] = sum_m dlogit[m] h7[m][j].
__global__ void k_dact_grad(const float *dH, const float *dlogit, const float *theta, const float *Z, int W,
                            const __nv_bfloat16 *h7, __nv_bfloat16 *dz, __nv_bfloat16 *dzt, float *grad, int64_t off_b,
                            int rows)
{
    __shared__ __nv_bfloat16 t[32][33];
    __shared__ float colsum[32], colw[32];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (ty == 0) {
        colsum[tx] = 0.f;
        colw[tx] = 0.f;
    }
    __syncthreads();
    float cs = 0.f, cw = 0.f;
    for (int k = ty; k < 32; k += 8) {
        const int m = r0 + k, j = c0 + tx;
        const int64_t e = (int64_t)m * W + j;
        const float z = Z[e];
        const float sg = sigm(z);
        const float dsilu = sg * (1.0f + z * (1.0f - sg));
        const float dh = dlogit ? dlogit[m] * theta[OFF_W8 + j] : dH[e];
        const float d = dh * dsilu;
        const __nv_bfloat16 db = __float2bfloat16_rn(d);
        dz[e] = db;
        t[k][tx] = db;
        cs += d;
        if (dlogit) cw = fmaf(dlogit[m], __bfloat162float(h7[e]), cw);
    }
    atomicAdd(&colsum[tx], cs);
    if (dlogit) atomicAdd(&colw[tx], cw);
    __syncthreads();
    for (int k = ty; k < 32; k += 8) dzt[(int64_t)(c0 + k) * rows + r0 + tx] = t[tx][k];
    if (ty == 0) {
        atomicAdd(&grad[off_b + c0 + tx], colsum[tx]);
        if (dlogit) atomicAdd(&grad[OFF_W8 + c0 + tx], colw[tx]);
    }
}

// Adam (Kingma and Ba 2015, bias-corrected, steps from 1) on the trainable entries;
// structural zeros get no gradient and so never move.
__global__ void k_dadam(float *theta, float *m, float *v, const float *grad, float lr, float b1t, float b2t)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = is_param(i) ? grad[i] : 0.f;
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / (1.f - b1t)) / (sqrtf(vi / (1.f - b2t)) + eps);
    }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct Ws {
    __nv_bfloat16 *wa, *wb, *w4, *w5, *w7, *wbt, *w4t, *w5t, *w7t;
    __nv_bfloat16 *ha, *h3, *h4, *h6, *h7;                       // activations [rows][width]
    __nv_bfloat16 *xt, *hat, *h3t, *h4t, *h6t, *dz, *dzt;        // training
    float *za, *zb, *z4, *z5, *z7, *dh, *grad, *dlogit;          // training
    size_t total;
};

Ws carve(char *base, int64_t rows, bool training)
{
    Ws w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    using bf = __nv_bfloat16;
    const size_t hb = sizeof(bf), fb = sizeof(float);
    w.wa = (bf *)take(hb * NA * IN);
    w.wb = (bf *)take(hb * NB * NA);
    w.w4 = (bf *)take(hb * NH * NH);
    w.w5 = (bf *)take(hb * NH * NH);
    w.w7 = (bf *)take(hb * NH * NH);
    w.ha = (bf *)take(hb * NA * rows);
    w.h3 = (bf *)take(hb * NH * rows);
    w.h4 = (bf *)take(hb * NH * rows);
    w.h6 = (bf *)take(hb * NH * rows);
    w.h7 = (bf *)take(hb * NH * rows);
    if (training) {
        w.wbt = (bf *)take(hb * NA * NB);
        w.w4t = (bf *)take(hb * NH * NH);
        w.w5t = (bf *)take(hb * NH * NH);
        w.w7t = (bf *)take(hb * NH * NH);
        w.xt = (bf *)take(hb * IN * rows);
        w.hat = (bf *)take(hb * NA * rows);
        w.h3t = (bf *)take(hb * NH * rows);
        w.h4t = (bf *)take(hb * NH * rows);
        w.h6t = (bf *)take(hb * NH * rows);
        w.dz = (bf *)take(hb * NA * rows);
        w.dzt = (bf *)take(hb * NA * rows);
        w.za = (float *)take(fb * NA * rows);
        w.zb = (float *)take(fb * NH * rows);
        w.z4 = (float *)take(fb * NH * rows);
        w.z5 = (float *)take(fb * NH * rows);
        w.z7 = (float *)take(fb * NH * rows);
        w.dh = (float *)take(fb * NA * rows);
        w.grad = (float *)take(fb * NPARAM);
        w.dlogit = (float *)take(fb * rows);
    }
    w.total = off;
    return w;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// One dense layer: out = act(A W^T + bias (+ Cadd)) with the optional outputs of GemmArgs.
GemmArgs layer(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *W, int M, int N, int K, const float *bias)
{
    GemmArgs g{};
    g.A = A;
    g.lda = lda;
    g.B = W;
    g.ldb = K;
    g.M = M;
    g.N = N;
    g.K = K;
    g.bias = bias;
    return g;
}

// The forward pass of `m` rows: x [m][IN] -> h7 [m][NH]; with `tr` the pre-activations
// and transposed activations that the backward pass reads are kept too.
cudaError_t forward_rows(const float *theta, const __nv_bfloat16 *x, int m, const Ws &w, bool tr, cudaStream_t s)
{
    cudaError_t e;
    GemmArgs g = layer(x, IN, w.wa, m, NA, IN, theta + OFF_BA);
    g.H = w.ha;
    g.ldh = NA;
    if (tr) {
        g.C = w.za, g.ldc = NA;
        g.Ht = w.hat, g.ldht = m;
    }
    if ((e = mlp::gemm(g, s)) != cudaSuccess) return e;
    g = layer(w.ha, NA, w.wb, m, NB, NA, theta + OFF_BB);
    g.H = w.h3;
    g.ldh = NH;
    if (tr) {
        g.C = w.zb, g.ldc = NH;
        g.Ht = w.h3t, g.ldht = m;
    }
    if ((e = mlp::gemm(g, s)) != cudaSuccess) return e;
    g = layer(w.h3, NH, w.w4, m, NH, NH, theta + OFF_B4);
    g.H = w.h4;
    g.ldh = NH;
    if (tr) {
        g.C = w.z4, g.ldc = NH;
        g.Ht = w.h4t, g.ldht = m;
    }
    if ((e = mlp::gemm(g, s)) != cudaSuccess) return e;
    g = layer(w.h4, NH, w.w5, m, NH, NH, theta + OFF_B5);  // h6 = h4 + SiLU(z5)
    g.R = w.h4;
    g.ldr = NH;
    g.H = w.h6;
    g.ldh = NH;
    if (tr) {
        g.C = w.z5, g.ldc = NH;
        g.Ht = w.h6t, g.ldht = m;
    }
    if ((e = mlp::gemm(g, s)) != cudaSuccess) return e;
    g = layer(w.h6, NH, w.w7, m, NH, NH, theta + OFF_B7);
    g.H = w.h7;
    g.ldh = NH;
    if (tr) g.C = w.z7, g.ldc = NH;
    return mlp::gemm(g, s);
}

}  // namespace dual
}  // namespace psa

using namespace psa::dual;

extern "C" {

int psa_dual_workspace_bytes(int64_t rows, int32_t training, size_t *bytes)
{
    if (rows < 0 || !bytes) return PSA_EINVAL;
    const int64_t r = training ? rows : (rows < FWD_CHUNK ? rows : FWD_CHUNK);
    *bytes = carve(nullptr, (r + TILE - 1) / TILE * TILE, training != 0).total;
    return PSA_OK;
}

int psa_dual_forward(const float *theta, const uint16_t *x, int64_t rows, float *prob, void *workspace,
                     size_t ws_bytes, void *stream_ptr)
{
    if (!theta || rows < 0 || (rows > 0 && (!x || !prob)) || !aligned16(x)) return PSA_EINVAL;
    size_t need = 0;
    psa_dual_workspace_bytes(rows, 0, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return PSA_EWORKSPACE;
    if (rows == 0) return PSA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream_ptr);
    const int64_t chunk = rows < FWD_CHUNK ? rows : FWD_CHUNK;
    const Ws w = carve(static_cast<char *>(workspace), (chunk + TILE - 1) / TILE * TILE, false);
    k_dshadow<<<256, 256, 0, s>>>(theta, w.wa, w.wb, w.w4, w.w5, w.w7, nullptr, nullptr, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    const __nv_bfloat16 *xb = reinterpret_cast<const __nv_bfloat16 *>(x);
    for (int64_t r0 = 0; r0 < rows; r0 += FWD_CHUNK) {
        const int m = (int)(rows - r0 < FWD_CHUNK ? rows - r0 : FWD_CHUNK);
        if (forward_rows(theta, xb + r0 * IN, m, w, false, s) != cudaSuccess) return PSA_ECUDA;
        const int64_t threads = (int64_t)m * 32;
        k_dhead<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(w.h7, theta, prob + r0, m);
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    }
    return PSA_OK;
}

int psa_dual_train_step(float *theta, float *adam_m, float *adam_v, int32_t step, float lr, const uint16_t *x,
                        const float *y, int64_t rows, float *loss, void *workspace, size_t ws_bytes, void *stream_ptr)
{
    if (!theta || !adam_m || !adam_v || !x || !y || !loss || step < 1 || !(lr > 0.f) || rows < TILE ||
        rows % TILE || rows > (1 << 24) || !aligned16(x))
        return PSA_EINVAL;
    size_t need = 0;
    psa_dual_workspace_bytes(rows, 1, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return PSA_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream_ptr);
    const Ws w = carve(static_cast<char *>(workspace), rows, true);
    const int B = (int)rows;
    const __nv_bfloat16 *xb = reinterpret_cast<const __nv_bfloat16 *>(x);
    if (cudaMemsetAsync(w.grad, 0, sizeof(float) * NPARAM, s) != cudaSuccess) return PSA_ECUDA;
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return PSA_ECUDA;
    k_dshadow<<<256, 256, 0, s>>>(theta, w.wa, w.wb, w.w4, w.w5, w.w7, w.wbt, w.w4t, w.w5t, w.w7t);
    k_dtranspose<<<dim3(B / 32, IN / 32), dim3(32, 8), 0, s>>>(xb, w.xt, B);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    if (forward_rows(theta, xb, B, w, true, s) != cudaSuccess) return PSA_ECUDA;
    k_dhead_train<<<(B * 32 + 255) / 256, 256, 0, s>>>(w.h7, theta, y, w.dlogit, w.grad, loss, B);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;

    const dim3 tb(32, 8);
    // weight gradient dW = dZ^T X: [out x B] * ([in x B])^T into grad + off (row-major [out][in])
    auto wgrad = [&](int out, int in, const __nv_bfloat16 *xin_t, int64_t off) {
        GemmArgs d = layer(w.dzt, B, xin_t, out, in, B, nullptr);
        d.ldb = B;
        d.C = w.grad + off;
        d.ldc = in;
        return psa::mlp::gemm(d, s);
    };
    // input gradient dH = dZ W: [B x out] * (W^T [in x out])^T into w.dh (+ Cadd)
    auto igrad = [&](int out, int in, const __nv_bfloat16 *wt, const float *cadd) {
        GemmArgs e = layer(w.dz, out, wt, B, in, out, nullptr);
        e.Cadd = cadd;
        e.ldcadd = in;
        e.C = w.dh;
        e.ldc = in;
        return psa::mlp::gemm(e, s);
    };
    // projection layer 7 (dh from the output unit)
    k_dact_grad<<<dim3(B / 32, NH / 32), tb, 0, s>>>(nullptr, w.dlogit, theta, w.z7, NH, w.h7, w.dz, w.dzt, w.grad,
                                                     OFF_B7, B);
    if (cudaGetLastError() != cudaSuccess || wgrad(NH, NH, w.h6t, OFF_W7) != cudaSuccess ||
        igrad(NH, NH, w.w7t, nullptr) != cudaSuccess)
        return PSA_ECUDA;
    // layer 5: h6 = h4 + h5, so dh5 = dh6 and dh4 = dh6 + W5^T dz5 (the add rides in the epilogue)
    k_dact_grad<<<dim3(B / 32, NH / 32), tb, 0, s>>>(w.dh, nullptr, theta, w.z5, NH, nullptr, w.dz, w.dzt, w.grad,
                                                     OFF_B5, B);
    if (cudaGetLastError() != cudaSuccess || wgrad(NH, NH, w.h4t, OFF_W5) != cudaSuccess ||
        igrad(NH, NH, w.w5t, w.dh) != cudaSuccess)
        return PSA_ECUDA;
    // layer 4
    k_dact_grad<<<dim3(B / 32, NH / 32), tb, 0, s>>>(w.dh, nullptr, theta, w.z4, NH, nullptr, w.dz, w.dzt, w.grad,
                                                     OFF_B4, B);
    if (cudaGetLastError() != cudaSuccess || wgrad(NH, NH, w.h3t, OFF_W4) != cudaSuccess ||
        igrad(NH, NH, w.w4t, nullptr) != cudaSuccess)
        return PSA_ECUDA;
    // layer B (the two pathways' second layers)
    k_dact_grad<<<dim3(B / 32, NB / 32), tb, 0, s>>>(w.dh, nullptr, theta, w.zb, NB, nullptr, w.dz, w.dzt, w.grad,
                                                     OFF_BB, B);
    if (cudaGetLastError() != cudaSuccess || wgrad(NB, NA, w.hat, OFF_WB) != cudaSuccess ||
        igrad(NB, NA, w.wbt, nullptr) != cudaSuccess)
        return PSA_ECUDA;
    // layer A (the two pathways' first layers)
    k_dact_grad<<<dim3(B / 32, NA / 32), tb, 0, s>>>(w.dh, nullptr, theta, w.za, NA, nullptr, w.dz, w.dzt, w.grad,
                                                     OFF_BA, B);
    if (cudaGetLastError() != cudaSuccess || wgrad(NA, IN, w.xt, OFF_WA) != cudaSuccess) return PSA_ECUDA;

    const float b1t = powf(0.9f, (float)step), b2t = powf(0.999f, (float)step);
    k_dadam<<<256, 256, 0, s>>>(theta, adam_m, adam_v, w.grad, lr, b1t, b2t);
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

}  // extern "C"
