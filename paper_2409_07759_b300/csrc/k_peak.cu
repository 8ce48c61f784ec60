// k_peak.cu -- FP32-pipe throughput probe, the denominator of the blends'
// roofline (they are arithmetic-bound: no tensor cores, little DRAM traffic).
//
// Every thread runs kChains independent multiply-add chains for `iters`
// iterations, either as scalar FP32 FMAs or as packed FP32x2 FMAs
// (__ffma2_rn, two FMAs per instruction), so that the issue rate rather than
// the FMA latency bounds the launch. The chains' sum is written to a sink, so
// nothing is optimised away. FLOPs of a launch = threads x iters x kChains x
// (2 per FMA) x (2 lanes when packed).
#include "swgs_internal.cuh"

namespace swgs {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads)
fp32_peak_kernel(int iters, float mul, float add, float* __restrict__ sink) {
    const int t = blockIdx.x * kPeakThreads + threadIdx.x;
    float out = 0.f;
    if constexpr (PACKED) {
        float2 a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            a[k] = make_float2(1e-3f * (float)(t & 1023) + (float)k, (float)k - 1e-3f * (float)(t & 511));
        const float2 m = make_float2(mul, mul), c = make_float2(add, add);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) out += a[k].x + a[k].y;
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)(t & 1023) + (float)k;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], mul, add);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) out += a[k];
    }
    sink[t] = out;
}

}  // namespace

}  // namespace swgs

using namespace swgs;

extern "C" swgs_status swgs_fp32_peak_launch(int32_t packed, int32_t blocks, int32_t iters,
                                             float* sink, double* flops, void* stream) {
    if ((packed != 0 && packed != 1) || blocks <= 0 || iters <= 0 || !sink || !flops)
        return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    note_launch();
    // mul slightly below 1 and a small add keep every chain finite and normal
    if (packed)
        fp32_peak_kernel<true><<<blocks, kPeakThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
    else
        fp32_peak_kernel<false><<<blocks, kPeakThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
    if (cudaGetLastError() != cudaSuccess) return SWGS_ECUDA;
    *flops = (double)blocks * kPeakThreads * (double)iters * kChains * 2.0 * (packed ? 2.0 : 1.0);
    return SWGS_OK;
}
