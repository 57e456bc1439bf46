// Throughput probes of the arithmetic pipes the assembly and right-hand side
// run on (no counterpart in the paper; they give the measured denominators of
// the roofline fractions).  Every thread runs kChains independent dependency
// chains of one instruction kind, so the pipe, not latency, sets the rate:
//   FP32 FMA      a = a * b + c                  (2 flop per instruction)
//   MUFU lg2      a = lg2.approx(a) + 1          (a stays in [1, 2); the add
//                 goes to the FMA pipe, which has 8x the lanes of the MUFU)
//   MUFU rcp      a = rcp.approx(a) + 1/2        (a tends to the fixed point 1.28;
//                 the add keeps successive reciprocals from cancelling)
//   FP64 FMA      a = a * b + c                  (2 flop per instruction)
// The grid fills every SM (resident blocks per SM from the occupancy query);
// the result is counted instructions (flop for the FMA kinds) per second of
// one launch timed with CUDA events after a warm-up launch.
#include "igs_internal.h"

namespace igs {

constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) k_peak(int iters, float seed, float* __restrict__ sink) {
    float a[kChains];
    double ad[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        a[c] = 1.0f + 0.1f * (float)((threadIdx.x + c) & 7) * seed;
        ad[c] = (double)a[c];
    }
    const float b = 0.999f, cc = 1e-3f * seed;
    const double bd = 0.999, cd = 1e-3 * (double)seed;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == IGS_PEAK_FP32_FMA) {
                    a[c] = fmaf(a[c], b, cc);
                } else if (KIND == IGS_PEAK_MUFU_LG2) {
                    float r;
                    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
                    a[c] = r + 1.0f;
                } else if (KIND == IGS_PEAK_MUFU_RCP) {
                    float r;
                    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
                    a[c] = r + 0.5f;
                } else {
                    ad[c] = fma(ad[c], bd, cd);
                }
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += (KIND == IGS_PEAK_FP64_FMA) ? (float)ad[c] : a[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;     // keeps the chains live; never true in practice
}

template <int KIND>
static double run_peak(int device, double* ms_out) {
    int sms = 0, per = 0;
    IGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    IGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_peak<KIND>, 256, 0));
    per = std::max(per, 1);
    const int grid = sms * per;
    // about 20-50 ms per launch on this class of GPU
    const int iters = (KIND == IGS_PEAK_FP64_FMA) ? 256 : (KIND == IGS_PEAK_FP32_FMA ? 16384 : 2048);
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double rate = 0.0;
    IGS_CUDA(cudaMalloc(&sink, 256 * sizeof(float)));
    try {
        IGS_CUDA(cudaEventCreate(&e0));
        IGS_CUDA(cudaEventCreate(&e1));
        k_peak<KIND><<<grid, 256>>>(iters, 1.0f, sink);          // warm-up
        IGS_CUDA(cudaGetLastError());
        IGS_CUDA(cudaEventRecord(e0));
        k_peak<KIND><<<grid, 256>>>(iters, 1.0f, sink);
        IGS_CUDA(cudaEventRecord(e1));
        IGS_CUDA(cudaGetLastError());
        IGS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        IGS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double insts = (double)grid * 256.0 * iters * 16.0 * kChains;
        const double per_inst = (KIND == IGS_PEAK_FP32_FMA || KIND == IGS_PEAK_FP64_FMA) ? 2.0 : 1.0;
        rate = insts * per_inst / (ms * 1e-3);
        if (ms_out) *ms_out = ms;
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(sink);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return rate;
}

double measure_peak(int device, int kind, double* ms) {
    IGS_CUDA(cudaSetDevice(device));
    switch (kind) {
        case IGS_PEAK_FP32_FMA: return run_peak<IGS_PEAK_FP32_FMA>(device, ms);
        case IGS_PEAK_MUFU_LG2: return run_peak<IGS_PEAK_MUFU_LG2>(device, ms);
        case IGS_PEAK_MUFU_RCP: return run_peak<IGS_PEAK_MUFU_RCP>(device, ms);
        case IGS_PEAK_FP64_FMA: return run_peak<IGS_PEAK_FP64_FMA>(device, ms);
        default: throw Error(IGS_E_INVALID_ARG, "unknown peak kind");
    }
}

}  // namespace igs
