// FP32 fused multiply-add throughput of the GPU: the denominator of the
// force sweep's roofline (an ALU-bound kernel), measured on the device
// instead of derived from the unit counts and the clock.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lc.h"
#include "lc_internal.cuh"

namespace lc {

constexpr int kProbeChains = 8;   // independent FMA chains per thread (hides the pipe latency)

// Every thread runs kProbeChains chains of packed f32x2 FMAs (two FMAs, four
// flops per instruction).  The values stay bounded (v <- v * m + c with
// |m| < 1) and are kept live by a store that depends on them.
__global__ void __launch_bounds__(256) k_ffma2_probe(float2 *out, int iters, float seed) {
    float2 v[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k)
        v[k] = make_float2(seed * (float)(threadIdx.x + k), seed * (float)(blockIdx.x + k));
    const float2 m = make_float2(0.999f, 0.998f), c = make_float2(1.0e-3f, 2.0e-3f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) v[k] = __ffma2_rn(v[k], m, c);
    }
    float2 s = v[0];
#pragma unroll
    for (int k = 1; k < kProbeChains; ++k) s = __fadd2_rn(s, v[k]);
    if (s.x == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains
}

}  // namespace lc

using namespace lc;

extern "C" lc_status lc_probe_fp32(int32_t iters, double *flops, double *seconds, void *stream) {
    if (iters <= 0 || !flops || !seconds) return LC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) { cudaGetLastError(); return LC_ERR_CUDA; }
    const int blocks = sms * 8, threads = 256;   // 64 warps per SM
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return LC_ERR_CUDA;
    }
    k_ffma2_probe<<<blocks, threads, 0, s>>>(nullptr, iters / 16 > 0 ? iters / 16 : 1, 1.0e-6f);   // warm-up
    cudaEventRecord(e0, s);
    k_ffma2_probe<<<blocks, threads, 0, s>>>(nullptr, iters, 1.0e-6f);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    if (!e) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) { cudaGetLastError(); return LC_ERR_CUDA; }
    *flops = 4.0 * kProbeChains * (double)iters * (double)blocks * (double)threads;
    *seconds = 1.0e-3 * (double)ms;
    return LC_OK;
}
