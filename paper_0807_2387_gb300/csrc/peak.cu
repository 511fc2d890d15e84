// Arithmetic throughput probes: the denominators of the roofline fractions of the
// ALU-bound kernels (the near field, the spreading and the interpolation), measured on
// the GPU the library runs on instead of taken from a nominal formula.
//
// Each thread runs kChains independent dependency chains so that the pipe, not the
// latency of one chain, is the limit; the grid is a multiple of the SM count and keeps
// 32 warps per SM resident.  Modes:
//   FS_PROBE_FFMA   scalar FP32 fused multiply-add (2 flop per lane)
//   FS_PROBE_FFMA2  packed two-wide FP32 fma (__ffma2_rn: 4 flop per lane)
//   FS_PROBE_MUFU   single MUFU operations (rcp.approx and lg2.approx on alternate chains, each
//                   followed by an add so that no pair of them folds: 1 op per lane)
// Work per launch = threads x iters x kChains x (ops per lane per chain step), timed with
// CUDA events around `reps` back-to-back launches after one warm-up launch.
#include <cuda_runtime.h>

#include "internal.h"
#include "plan.h"

namespace fs {

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

__device__ __forceinline__ float probe_rcp(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float probe_lg2(float x)
{
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int MODE> __global__ void __launch_bounds__(kProbeThreads) k_probe(int iters, float a, float b, float *out)
{
    float2 v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        v[k] = make_float2(1.0f + 1e-3f * (float)(threadIdx.x + k), 2.0f - 1e-3f * (float)k);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if constexpr (MODE == FS_PROBE_FFMA) {
                v[k].x = fmaf(v[k].x, a, b);
                v[k].y = fmaf(v[k].y, a, b);
            } else if constexpr (MODE == FS_PROBE_FFMA2) {
                v[k] = __ffma2_rn(v[k], a2, b2);
            } else if (k % 2 == 0) {
                v[k].x = probe_rcp(v[k].x) + 1.0f;   // fixed point (1 + sqrt 5) / 2
            } else {
                v[k].x = probe_lg2(v[k].x) + 2.0f;   // fixed point 4
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        s += v[k].x + v[k].y;
    if (s == 1234.5f)   // practically never true; keeps the chains live
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace fs

extern "C" {

fs_status fs_probe_throughput(int mode, int iters, int reps, double *ops_per_s, double *ms_per_launch)
{
    using namespace fs;
    if (!ops_per_s || !ms_per_launch)
        return fail(FS_EINVAL, "null argument");
    if (mode != FS_PROBE_FFMA && mode != FS_PROBE_FFMA2 && mode != FS_PROBE_MUFU)
        return fail(FS_EINVAL, "unknown probe mode");
    if (iters < 1 || reps < 1)
        return fail(FS_EINVAL, "iters and reps must be >= 1");
    int dev = 0, sms = 0;
    FS_CUDA(cudaGetDevice(&dev));
    FS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)(sms * kProbeBlocksPerSm);
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc(&out, sizeof(float) * blocks * kProbeThreads);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    auto launch = [&]() {
        if (mode == FS_PROBE_FFMA)
            k_probe<FS_PROBE_FFMA><<<blocks, kProbeThreads, 0, st>>>(iters, 0.999999f, 1e-6f, out);
        else if (mode == FS_PROBE_FFMA2)
            k_probe<FS_PROBE_FFMA2><<<blocks, kProbeThreads, 0, st>>>(iters, 0.999999f, 1e-6f, out);
        else
            k_probe<FS_PROBE_MUFU><<<blocks, kProbeThreads, 0, st>>>(iters, 0.f, 0.f, out);
        return cudaGetLastError();
    };
    if (e == cudaSuccess)
        e = launch();   // warm-up
    if (e == cudaSuccess)
        e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = launch();
    if (e == cudaSuccess)
        e = cudaEventRecord(e1, st);
    if (e == cudaSuccess)
        e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (out)
        cudaFree(out);
    if (st)
        cudaStreamDestroy(st);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, std::string("throughput probe: ") + cudaGetErrorString(e));
    const double per_lane = mode == FS_PROBE_FFMA ? 2.0 * 2.0 : (mode == FS_PROBE_FFMA2 ? 4.0 : 1.0);
    const double ops = (double)blocks * kProbeThreads * (double)iters * kChains * per_lane * reps;
    *ms_per_launch = (double)ms / reps;
    *ops_per_s = ops / ((double)ms * 1e-3);
    return FS_OK;
}

}  // extern "C"
