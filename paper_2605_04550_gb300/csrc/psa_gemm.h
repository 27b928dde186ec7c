// psa_gemm.h -- the tensor-core GEMM of the classifier kernels (psa_mlp.cu), shared
// by the two networks of the learned restriction (not public).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace psa {
namespace mlp {

constexpr int TILE = 128;  // M and N of a CTA tile
constexpr int KCH = 64;    // K per shared-memory chunk (4 MMAs of K = 16)

// C[M x N] = A[M x K] * B[N x K]^T + bias on the tensor cores (BF16 operands, K
// contiguous, FP32 accumulation); N a multiple of TILE, K of KCH. Epilogue per
// element: z = acc + bias[col] + Cadd[row][col] (each optional); C = z; with
// a = silu(z) + R[row][col] (R optional), H = bf16(a) and Ht its transpose.
struct GemmArgs {
    const __nv_bfloat16 *A;
    int64_t lda;
    const __nv_bfloat16 *B;
    int64_t ldb;
    int M, N, K;
    const float *bias;      // [N] or null
    const float *Cadd;      // FP32 [M][ldcadd] added to the accumulator, or null
    int64_t ldcadd;
    float *C;               // FP32 z, row-major, ldc; or null
    int64_t ldc;
    const __nv_bfloat16 *R; // BF16 residual [M][ldr] added after the activation, or null
    int64_t ldr;
    __nv_bfloat16 *H;       // BF16 silu(z) (+ R), row-major, ldh; or null
    int64_t ldh;
    __nv_bfloat16 *Ht;      // the same, transposed ([N][M]), ldht; or null
    int64_t ldht;
};

// Launch on stream s (asynchronous; a tile whose bounded waits run out writes NaN
// and is counted for psa_mlp_timeouts).
cudaError_t gemm(const GemmArgs &g, cudaStream_t s);

}  // namespace mlp
}  // namespace psa
