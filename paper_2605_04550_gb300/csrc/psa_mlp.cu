// psa_mlp.cu -- the classifier of the restricted method: a multilayer
// perceptron with three hidden layers of 256 SiLU units and a sigmoid output
// (the paper's network maps per-point features to the probability that the
// point is sensitive, Sec. 3.2; its training uses binary cross-entropy and
// Adam, Sec. 3.4). Dense layers run as BF16 GEMMs on the tensor cores with FP32
// accumulation in tensor memory (tcgen05); bias, activation, loss and the
// optimiser run on the CUDA cores.
//
// GEMM: C[M x N] = A[M x K] * B[N x K]^T, A and B row-major BF16 (K contiguous,
// "K-major"). One CTA of 128 threads computes a 128 x 128 tile of C. Per K
// chunk of 64, TMA copies the A and B tiles (128 rows x 128 bytes each) into one
// of three shared-memory stages with the 128-byte swizzle; one thread issues
// four 128 x 128 x 16 MMAs into a 128-column FP32 accumulator in tensor memory
// once the stage's transaction barrier completes, commits them to the stage's
// second barrier, and refills the stage of the previous chunk as soon as its
// MMAs are done, so copies run two chunks ahead of the tensor core. The epilogue
// reads the accumulator with tcgen05.ld (warp w owns rows 32w .. 32w + 31),
// adds the bias and writes any of: FP32 pre-activation, BF16 SiLU output,
// BF16 SiLU output transposed (for the weight-gradient GEMMs of training).
#include <atomic>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mutex>

#include "psa.h"
#include "psa_gemm.h"
#include "psa_tc.cuh"

namespace psa {
namespace mlp {

constexpr int IN = PSA_MLP_IN;
constexpr int HID = PSA_MLP_HIDDEN;
// parameter vector (float32): W1[HID][IN], b1[HID], W2[HID][HID], b2[HID],
// W3[HID][HID], b3[HID], w4[HID], b4
constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + (int64_t)HID * IN;
constexpr int64_t OFF_W2 = OFF_B1 + HID;
constexpr int64_t OFF_B2 = OFF_W2 + (int64_t)HID * HID;
constexpr int64_t OFF_W3 = OFF_B2 + HID;
constexpr int64_t OFF_B3 = OFF_W3 + (int64_t)HID * HID;
constexpr int64_t OFF_W4 = OFF_B3 + HID;
constexpr int64_t OFF_B4 = OFF_W4 + HID;
constexpr int64_t NPARAM = OFF_B4 + 1;
static_assert(NPARAM == PSA_MLP_PARAMS, "parameter count");

constexpr int TILE_BYTES = TILE * KCH * 2;
constexpr int STAGE_BYTES = 2 * TILE_BYTES;  // A and B tiles of one K chunk
constexpr int STAGES = 3;
// stages + barriers + TMEM slot + 1 KB for aligning the stages to the swizzle atom:
// 98 KB keeps <= 2 CTAs (256 TMEM columns) per SM
constexpr int GEMM_SMEM = STAGES * STAGE_BYTES + 2048;
constexpr int WAIT_LIMIT = 1 << 20;
constexpr int64_t FWD_CHUNK = 131072;  // rows per forward pass through the workspace

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }

// CTAs of k_gemm_bf16 whose bounded waits ran out since the last psa_mlp_timeouts
// call (their outputs are NaN; the host learns of them through that call).
__device__ unsigned int g_gemm_timeouts;

__global__ void __launch_bounds__(128) k_gemm_bf16(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB, const GemmArgs g)
{
    extern __shared__ unsigned char smem_raw[];
    // stages of (A tile, B tile) on 1024-byte boundaries (the swizzle atom), then the
    // barriers and the TMEM slot
    unsigned char *const smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *const full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *const empty = full + STAGES;
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(empty + STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TILE, n0 = blockIdx.y * TILE;
    const int nk = g.K / KCH;

    if (warp == 0) tc::tmem_alloc(tslot, TILE);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(TILE, TILE);

    // Thread 0 runs the pipeline: TMA loads of K chunk c into stage c % STAGES
    // complete on full[stage]; the chunk's four MMAs commit to empty[stage]; a stage is
    // loaded again once the MMAs that read it have completed.
    bool ok = true;
    if (tid == 0) {
        auto issue = [&](int c) {
            unsigned char *const sA = smem + (c % STAGES) * STAGE_BYTES;
            tc::mbar_arrive_expect_tx(&full[c % STAGES], STAGE_BYTES);
            tc::tma_load_2d(sA, &tmA, c * KCH, m0, &full[c % STAGES]);
            tc::tma_load_2d(sA + TILE_BYTES, &tmB, c * KCH, n0, &full[c % STAGES]);
        };
        for (int c = 0; c < nk && c < STAGES; ++c) issue(c);
        for (int c = 0; c < nk && ok; ++c) {
            const int st = c % STAGES;
            const uint32_t par = (uint32_t)((c / STAGES) & 1);
            if (!tc::mbar_wait(&full[st], par, WAIT_LIMIT)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint32_t a_base = tc::smem_addr(smem + st * STAGE_BYTES), b_base = a_base + TILE_BYTES;
#pragma unroll
            for (int s = 0; s < KCH / 16; ++s)
                tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + s * 32), tc::smem_desc_sw128(b_base + s * 32), IDESC,
                             (c > 0 || s > 0) ? 1u : 0u);
            tc::mma_commit(&empty[st]);
            // refill the stage of chunk c - 1 (its MMAs are queued ahead of chunk c's)
            const int r = c - 1 + STAGES;
            if (c >= 1 && r < nk) {
                const int sp = (c - 1) % STAGES;
                if (!tc::mbar_wait(&empty[sp], (uint32_t)(((c - 1) / STAGES) & 1), WAIT_LIMIT)) {
                    ok = false;
                    break;
                }
                issue(r);
            }
        }
    }
    // everyone waits for the last chunk's commit, which covers every MMA issued before it
    {
        const int last = nk - 1;
        bool done = true;
        if (last >= 0) {
            done = tc::mbar_wait(&empty[last % STAGES], (uint32_t)((last / STAGES) & 1), WAIT_LIMIT);
            if (!done) done = tc::mbar_wait(&empty[last % STAGES], (uint32_t)((last / STAGES) & 1), WAIT_LIMIT);
        }
        ok = __syncthreads_and((done && ok) ? 1 : 0) != 0;
    }
    if (!ok && tid == 0) atomicAdd(&g_gemm_timeouts, 1u);
    tc::fence_after_sync();

    // epilogue: thread = row m0 + 32 warp + lane, 32 columns per tensor-memory load
    const int row = m0 + 32 * warp + lane;
    const float qnan = __int_as_float(0x7fc00000);
#pragma unroll 1
    for (int c0 = 0; c0 < TILE; c0 += 32) {
        uint32_t r[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
        if (row >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            float z = ok ? __uint_as_float(r[j]) : qnan;  // a timed-out wait leaves NaN
            if (g.bias) z += g.bias[col];
            if (g.Cadd) z += g.Cadd[(int64_t)row * g.ldcadd + col];
            if (g.C) g.C[(int64_t)row * g.ldc + col] = z;
            if (g.H || g.Ht) {
                float a = silu(z);
                if (g.R) a += __bfloat162float(g.R[(int64_t)row * g.ldr + col]);
                const __nv_bfloat16 h = __float2bfloat16_rn(a);
                if (g.H) g.H[(int64_t)row * g.ldh + col] = h;
                if (g.Ht) g.Ht[(int64_t)col * g.ldht + row] = h;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TILE);
    }
}

constexpr int kMaxDevices = 64;
std::atomic<bool> g_attr_set[kMaxDevices];

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
std::once_flag g_encode_once;
EncodeTiledFn g_encode = nullptr;

EncodeTiledFn encode_fn()
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    });
    return g_encode;
}

// Tensor map of a row-major BF16 matrix [rows][cols] (leading dimension ld elements)
// read in 128 x 64 boxes with the 128-byte swizzle; rows past the end read as zero.
cudaError_t tile_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t rows, int64_t cols, int64_t ld)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)KCH, (cuuint32_t)TILE};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t gemm(const GemmArgs &g, cudaStream_t s)
{
    // the dynamic shared-memory limit is a per-device attribute of the kernel
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_attr_set[dev].load()) {
        e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
        if (e != cudaSuccess) return e;
        g_attr_set[dev].store(true);
    }
    CUtensorMap ta, tb;
    if ((e = tile_map(&ta, g.A, g.M, g.K, g.lda)) != cudaSuccess) return e;
    if ((e = tile_map(&tb, g.B, g.N, g.K, g.ldb)) != cudaSuccess) return e;
    const dim3 grid((unsigned)((g.M + TILE - 1) / TILE), (unsigned)(g.N / TILE));
    k_gemm_bf16<<<grid, 128, GEMM_SMEM, s>>>(ta, tb, g);
    return cudaGetLastError();
}

// -------------------------------------------------------------- elementwise
// BF16 copies of the weight matrices: W (as stored, [out][in]) and, for
// training, W^T ([in][out]).
__global__ void k_shadow(const float *theta, __nv_bfloat16 *w1, __nv_bfloat16 *w2, __nv_bfloat16 *w3,
                         __nv_bfloat16 *w2t, __nv_bfloat16 *w3t)
{
    const int64_t n1 = (int64_t)HID * IN, n2 = (int64_t)HID * HID;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1 + 2 * n2; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n1) {
            w1[i] = __float2bfloat16_rn(theta[OFF_W1 + i]);
            continue;
        }
        const int64_t q = (i - n1) % n2;
        const bool second = (i - n1) < n2;
        const float v = theta[(second ? OFF_W2 : OFF_W3) + q];
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        (second ? w2 : w3)[q] = b;
        __nv_bfloat16 *t = second ? w2t : w3t;
        if (t) {
            const int64_t o = q / HID, in = q % HID;
            t[in * HID + o] = b;
        }
    }
}

// x^T ([IN][rows]) of a batch, for the first layer's weight gradient.
__global__ void k_transpose_in(const __nv_bfloat16 *x, __nv_bfloat16 *xt, int rows)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) t[k][threadIdx.x] = x[(int64_t)(r0 + k) * IN + c0 + threadIdx.x];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) xt[(int64_t)(c0 + k) * rows + r0 + threadIdx.x] = t[threadIdx.x][k];
}

// Output unit: prob = sigmoid(h3 . w4 + b4), one warp per row.
__global__ void k_head(const __nv_bfloat16 *h3, const float *theta, float *prob, int64_t rows)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const uint4 v = *reinterpret_cast<const uint4 *>(h3 + row * HID + lane * 8);
    const __nv_bfloat16 *hb = reinterpret_cast<const __nv_bfloat16 *>(&v);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s = fmaf(__bfloat162float(hb[j]), theta[OFF_W4 + lane * 8 + j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) prob[row] = 1.0f / (1.0f + __expf(-(s + theta[OFF_B4])));
}

// Training output unit: logit, mean binary cross-entropy (added to *loss) and
// dL/dlogit = (sigmoid(logit) - y) / rows; d b4 accumulated into grad.
__global__ void k_head_train(const __nv_bfloat16 *h3, const float *theta, const float *y, float *dlogit, float *grad,
                             float *loss, int rows)
{
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const uint4 v = *reinterpret_cast<const uint4 *>(h3 + (int64_t)row * HID + lane * 8);
    const __nv_bfloat16 *hb = reinterpret_cast<const __nv_bfloat16 *>(&v);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s = fmaf(__bfloat162float(hb[j]), theta[OFF_W4 + lane * 8 + j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const float l = s + theta[OFF_B4];
        const float t = y[row];
        // stable BCE with logits: max(l, 0) - l t + log(1 + exp(-|l|))
        const float bce = fmaxf(l, 0.f) - l * t + log1pf(__expf(-fabsf(l)));
        const float p = 1.0f / (1.0f + __expf(-l));
        const float d = (p - t) / (float)rows;
        dlogit[row] = d;
        atomicAdd(loss, bce / (float)rows);
        atomicAdd(&grad[OFF_B4], d);
    }
}

// Backward through one SiLU layer on a 32 x 32 tile: dz = dh * silu'(z) with
// dh = dH[m][j] (dlogit != null: dh = dlogit[m] * w4[j]); writes dz (BF16, row-major
// and transposed), adds the bias gradient sum_m dz into grad[off_b + j] and, for
// the last hidden layer, d w4[j] = sum_m dlogit[m] h3[m][j].
__global__ void k_act_grad(const float *dH, const float *dlogit, const float *theta, const float *Z,
                           const __nv_bfloat16 *h3, __nv_bfloat16 *dz, __nv_bfloat16 *dzt, float *grad, int64_t off_b,
                           int rows)
{
    __shared__ __nv_bfloat16 t[32][33];
    __shared__ float colsum[32], colw4[32];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (ty == 0) {
        colsum[tx] = 0.f;
        colw4[tx] = 0.f;
    }
    __syncthreads();
    float cs = 0.f, cw = 0.f;
    for (int k = ty; k < 32; k += 8) {
        const int m = r0 + k, j = c0 + tx;
        const int64_t e = (int64_t)m * HID + j;
        const float z = Z[e];
        const float sg = 1.0f / (1.0f + __expf(-z));
        const float dsilu = sg * (1.0f + z * (1.0f - sg));
        const float dh = dlogit ? dlogit[m] * theta[OFF_W4 + j] : dH[e];
        const float d = dh * dsilu;
        const __nv_bfloat16 db = __float2bfloat16_rn(d);
        dz[e] = db;
        t[k][tx] = db;
        cs += d;
        if (dlogit) cw = fmaf(dlogit[m], __bfloat162float(h3[e]), cw);
    }
    atomicAdd(&colsum[tx], cs);
    if (dlogit) atomicAdd(&colw4[tx], cw);
    __syncthreads();
    for (int k = ty; k < 32; k += 8) dzt[(int64_t)(c0 + k) * rows + r0 + tx] = t[tx][k];
    if (ty == 0) {
        atomicAdd(&grad[off_b + c0 + tx], colsum[tx]);
        if (dlogit) atomicAdd(&grad[OFF_W4 + c0 + tx], colw4[tx]);
    }
}

// Adam (Kingma and Ba 2015) with bias correction; step counts from 1.
__global__ void k_adam(float *theta, float *m, float *v, const float *grad, int64_t n, float lr, float b1t, float b2t)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / (1.f - b1t)) / (sqrtf(vi / (1.f - b2t)) + eps);
    }
}

// ---------------------------------------------------------------- workspace
size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct Ws {
    __nv_bfloat16 *w1, *w2, *w3, *w2t, *w3t, *h1, *h2, *h3, *xt, *h1t, *h2t, *dz, *dzt;
    float *z1, *z2, *z3, *dh, *grad, *dlogit;
    size_t total;
};

// rows: the rows of one pass (forward chunk or training batch)
Ws carve(char *base, int64_t rows, bool training)
{
    Ws w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t hb = sizeof(__nv_bfloat16), fb = sizeof(float);
    w.w1 = (__nv_bfloat16 *)take(hb * HID * IN);
    w.w2 = (__nv_bfloat16 *)take(hb * HID * HID);
    w.w3 = (__nv_bfloat16 *)take(hb * HID * HID);
    w.h1 = (__nv_bfloat16 *)take(hb * HID * rows);
    w.h2 = (__nv_bfloat16 *)take(hb * HID * rows);
    w.h3 = (__nv_bfloat16 *)take(hb * HID * rows);
    if (training) {
        w.w2t = (__nv_bfloat16 *)take(hb * HID * HID);
        w.w3t = (__nv_bfloat16 *)take(hb * HID * HID);
        w.xt = (__nv_bfloat16 *)take(hb * IN * rows);
        w.h1t = (__nv_bfloat16 *)take(hb * HID * rows);
        w.h2t = (__nv_bfloat16 *)take(hb * HID * rows);
        w.dz = (__nv_bfloat16 *)take(hb * HID * rows);
        w.dzt = (__nv_bfloat16 *)take(hb * HID * rows);
        w.z1 = (float *)take(fb * HID * rows);
        w.z2 = (float *)take(fb * HID * rows);
        w.z3 = (float *)take(fb * HID * rows);
        w.dh = (float *)take(fb * HID * rows);
        w.grad = (float *)take(fb * NPARAM);
        w.dlogit = (float *)take(fb * rows);
    }
    w.total = off;
    return w;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace mlp
}  // namespace psa

using namespace psa::mlp;

extern "C" {

int psa_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int32_t M, int32_t N, int32_t K,
                  float *C, int64_t ldc, void *stream)
{
    if (!A || !B || !C || M < 0 || N < 0 || K < 0) return PSA_EINVAL;
    if (N % TILE || K % KCH || lda < K || ldb < K || ldc < N || lda % 8 || ldb % 8) return PSA_EINVAL;
    if (!aligned16(A) || !aligned16(B)) return PSA_EINVAL;
    if (M == 0 || N == 0) return PSA_OK;
    if (K == 0) return cudaMemset2DAsync(C, sizeof(float) * ldc, 0, sizeof(float) * N, M,
                                         static_cast<cudaStream_t>(stream)) == cudaSuccess ? PSA_OK : PSA_ECUDA;
    GemmArgs g{};
    g.A = reinterpret_cast<const __nv_bfloat16 *>(A);
    g.lda = lda;
    g.B = reinterpret_cast<const __nv_bfloat16 *>(B);
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.C = C;
    g.ldc = ldc;
    return gemm(g, static_cast<cudaStream_t>(stream)) == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

int psa_mlp_timeouts(uint32_t *count)
{
    if (!count) return PSA_EINVAL;
    unsigned int v = 0;
    const unsigned int zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_gemm_timeouts, sizeof(v)) != cudaSuccess) return PSA_ECUDA;
    if (v && cudaMemcpyToSymbol(g_gemm_timeouts, &zero, sizeof(zero)) != cudaSuccess) return PSA_ECUDA;
    *count = v;
    return PSA_OK;
}

int psa_mlp_workspace_bytes(int64_t rows, int32_t training, size_t *bytes)
{
    if (rows < 0 || !bytes) return PSA_EINVAL;
    const int64_t r = training ? rows : (rows < FWD_CHUNK ? rows : FWD_CHUNK);
    *bytes = carve(nullptr, (r + TILE - 1) / TILE * TILE, training != 0).total;
    return PSA_OK;
}

int psa_mlp_forward(const float *theta, const uint16_t *x, int64_t rows, float *prob, void *workspace,
                    size_t ws_bytes, void *stream_ptr)
{
    if (!theta || rows < 0 || (rows > 0 && (!x || !prob)) || !aligned16(x)) return PSA_EINVAL;
    size_t need = 0;
    psa_mlp_workspace_bytes(rows, 0, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return PSA_EWORKSPACE;
    if (rows == 0) return PSA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream_ptr);
    const int64_t chunk = rows < FWD_CHUNK ? rows : FWD_CHUNK;
    const Ws w = carve(static_cast<char *>(workspace), (chunk + TILE - 1) / TILE * TILE, false);
    k_shadow<<<256, 256, 0, s>>>(theta, w.w1, w.w2, w.w3, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    const __nv_bfloat16 *xb = reinterpret_cast<const __nv_bfloat16 *>(x);
    for (int64_t r0 = 0; r0 < rows; r0 += chunk) {
        const int m = (int)((rows - r0) < chunk ? (rows - r0) : chunk);
        GemmArgs g{};
        g.M = m;
        g.N = HID;
        g.A = xb + r0 * IN;
        g.lda = IN;
        g.B = w.w1;
        g.ldb = IN;
        g.K = IN;
        g.bias = theta + OFF_B1;
        g.H = w.h1;
        g.ldh = HID;
        if (gemm(g, s) != cudaSuccess) return PSA_ECUDA;
        g.A = w.h1;
        g.lda = HID;
        g.B = w.w2;
        g.ldb = HID;
        g.K = HID;
        g.bias = theta + OFF_B2;
        g.H = w.h2;
        if (gemm(g, s) != cudaSuccess) return PSA_ECUDA;
        g.A = w.h2;
        g.B = w.w3;
        g.bias = theta + OFF_B3;
        g.H = w.h3;
        if (gemm(g, s) != cudaSuccess) return PSA_ECUDA;
        const int64_t threads = (int64_t)m * 32;
        k_head<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(w.h3, theta, prob + r0, m);
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
    }
    return PSA_OK;
}

int psa_mlp_train_step(float *theta, float *adam_m, float *adam_v, int32_t step, float lr, const uint16_t *x,
                       const float *y, int64_t rows, float *loss, void *workspace, size_t ws_bytes, void *stream_ptr)
{
    if (!theta || !adam_m || !adam_v || !x || !y || !loss || step < 1 || !(lr > 0.f) || rows < TILE ||
        rows % TILE || rows > (1 << 24) || !aligned16(x))
        return PSA_EINVAL;
    size_t need = 0;
    psa_mlp_workspace_bytes(rows, 1, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return PSA_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream_ptr);
    const Ws w = carve(static_cast<char *>(workspace), rows, true);
    const int B = (int)rows;
    const __nv_bfloat16 *xb = reinterpret_cast<const __nv_bfloat16 *>(x);
    if (cudaMemsetAsync(w.grad, 0, sizeof(float) * NPARAM, s) != cudaSuccess) return PSA_ECUDA;
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return PSA_ECUDA;
    k_shadow<<<256, 256, 0, s>>>(theta, w.w1, w.w2, w.w3, w.w2t, w.w3t);
    k_transpose_in<<<dim3(B / 32, IN / 32), dim3(32, 8), 0, s>>>(xb, w.xt, B);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;

    // forward, keeping pre-activations and transposed activations
    GemmArgs g{};
    g.M = B;
    g.N = HID;
    g.A = xb;
    g.lda = IN;
    g.B = w.w1;
    g.ldb = IN;
    g.K = IN;
    g.bias = theta + OFF_B1;
    g.C = w.z1;
    g.ldc = HID;
    g.H = w.h1;
    g.ldh = HID;
    g.Ht = w.h1t;
    g.ldht = B;
    if (gemm(g, s) != cudaSuccess) return PSA_ECUDA;
    g.A = w.h1;
    g.lda = HID;
    g.B = w.w2;
    g.ldb = HID;
    g.K = HID;
    g.bias = theta + OFF_B2;
    g.C = w.z2;
    g.H = w.h2;
    g.Ht = w.h2t;
    if (gemm(g, s) != cudaSuccess) return PSA_ECUDA;
    g.A = w.h2;
    g.B = w.w3;
    g.bias = theta + OFF_B3;
    g.C = w.z3;
    g.H = w.h3;
    g.Ht = nullptr;
    if (gemm(g, s) != cudaSuccess) return PSA_ECUDA;
    k_head_train<<<(B * 32 + 255) / 256, 256, 0, s>>>(w.h3, theta, y, w.dlogit, w.grad, loss, B);
    if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;

    // backward: layer 3, 2, 1
    const dim3 tg(B / 32, HID / 32), tb(32, 8);
    const float *Zs[3] = {w.z1, w.z2, w.z3};
    const int64_t offB[3] = {OFF_B1, OFF_B2, OFF_B3};
    const int64_t offW[3] = {OFF_W1, OFF_W2, OFF_W3};
    const __nv_bfloat16 *Hin_t[3] = {w.xt, w.h1t, w.h2t};  // layer inputs, transposed
    const __nv_bfloat16 *Wt[3] = {nullptr, w.w2t, w.w3t};
    for (int L = 2; L >= 0; --L) {
        k_act_grad<<<tg, tb, 0, s>>>(w.dh, L == 2 ? w.dlogit : nullptr, theta, Zs[L], w.h3, w.dz, w.dzt, w.grad,
                                     offB[L], B);
        if (cudaGetLastError() != cudaSuccess) return PSA_ECUDA;
        // dW_L = dZ^T * input: [HID x B] * ([in x B])^T
        GemmArgs d{};
        d.A = w.dzt;
        d.lda = B;
        d.B = Hin_t[L];
        d.ldb = B;
        d.M = HID;
        d.N = L == 0 ? IN : HID;
        d.K = B;
        d.C = w.grad + offW[L];
        d.ldc = d.N;
        if (gemm(d, s) != cudaSuccess) return PSA_ECUDA;
        if (L > 0) {
            // dH_{L-1} = dZ * W_L: [B x HID] * (W_L^T [in x HID])^T
            GemmArgs e{};
            e.A = w.dz;
            e.lda = HID;
            e.B = Wt[L];
            e.ldb = HID;
            e.M = B;
            e.N = HID;
            e.K = HID;
            e.C = w.dh;
            e.ldc = HID;
            if (gemm(e, s) != cudaSuccess) return PSA_ECUDA;
        }
    }
    const float b1t = powf(0.9f, (float)step), b2t = powf(0.999f, (float)step);
    k_adam<<<256, 256, 0, s>>>(theta, adam_m, adam_v, w.grad, NPARAM, lr, b1t, b2t);
    return cudaGetLastError() == cudaSuccess ? PSA_OK : PSA_ECUDA;
}

}  // extern "C"
