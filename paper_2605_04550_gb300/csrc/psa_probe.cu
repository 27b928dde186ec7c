// psa_probe.cu -- micro-benchmark of the FP64 unit: the rates behind the roofline of
// the FP64-bound sigma_min path and behind its one-lane-per-point layout. A launch puts
// exactly one block of `warps_per_sm` warps on every SM; each thread of the first
// `active_lanes` lanes of its warp runs `chains` independent chains of one operation,
// and the result is the rate in lane-operations per second. Comparing active_lanes =
// 32 with 1 shows what a warp instruction costs when few lanes are active; comparing
// chains = 1 with 8 and the warps per SM shows how much latency a scheduler hides.
#include <cstdint>
#include <cuda_runtime.h>

#include "psa.h"

namespace psa {
namespace {

__device__ double g_fp64_probe_sink;

// OP: 0 a = a * m + c (one DFMA), 1 a = a + c, 2 a = a * m, 3 a = m / a, 4 a = sqrt(a)
template <int OP, int CH>
__global__ void k_probe_fp64(int iters, int active, double m, double c)
{
    if ((int)(threadIdx.x & 31) >= active) return;
    double a[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = 1.0 + threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            if (OP == 0) a[k] = fma(a[k], m, c);
            else if (OP == 1) a[k] = a[k] + c;
            else if (OP == 2) a[k] = a[k] * m;
            else if (OP == 3) a[k] = m / a[k];
            else a[k] = sqrt(a[k]);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += a[k];
    if (s == 1.2345678e-300) g_fp64_probe_sink = s;  // keeps the chains live
}

// Dynamic shared memory that no second block fits beside (more than half of an SM's
// 228 KB): one launch of SM-count blocks then puts exactly one block on every SM.
constexpr int kOneBlockSmem = 120 * 1024;

template <int OP, int CH>
void launch(int blocks, int threads, int iters, int active, cudaStream_t st)
{
    cudaFuncSetAttribute(k_probe_fp64<OP, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOneBlockSmem);
    k_probe_fp64<OP, CH><<<blocks, threads, kOneBlockSmem, st>>>(iters, active, 1.0000001, 1e-9);
}

using LaunchFn = void (*)(int, int, int, int, cudaStream_t);

LaunchFn pick(int op, int chains)
{
    const bool c8 = chains == 8;
    switch (op) {
    case 0: return c8 ? &launch<0, 8> : &launch<0, 1>;
    case 1: return c8 ? &launch<1, 8> : &launch<1, 1>;
    case 2: return c8 ? &launch<2, 8> : &launch<2, 1>;
    case 3: return c8 ? &launch<3, 8> : &launch<3, 1>;
    case 4: return c8 ? &launch<4, 8> : &launch<4, 1>;
    default: return nullptr;
    }
}

}  // namespace
}  // namespace psa

extern "C" int psa_probe_fp64(int32_t op, int32_t warps_per_sm, int32_t active_lanes, int32_t chains, int32_t iters,
                              double *lane_ops_per_s, void *stream)
{
    if (op < 0 || op > 4 || warps_per_sm < 1 || warps_per_sm > 32 || active_lanes < 1 || active_lanes > 32 ||
        (chains != 1 && chains != 8) || iters < 1 || iters > (1 << 24) || !lane_ops_per_s)
        return PSA_EINVAL;
    const psa::LaunchFn fn = psa::pick(op, chains);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSA_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return PSA_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int threads = warps_per_sm * 32;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PSA_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PSA_ECUDA;
    }
    fn(sms, threads, iters < 64 ? iters : 64, active_lanes, st);  // warm-up
    cudaEventRecord(e0, st);
    fn(sms, threads, iters, active_lanes, st);
    cudaEventRecord(e1, st);
    int rc = PSA_OK;
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
        rc = PSA_ECUDA;
    else
        *lane_ops_per_s = (double)sms * threads / 32.0 * active_lanes * chains * (double)iters / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
