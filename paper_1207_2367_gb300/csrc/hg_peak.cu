// hg_peak.cu -- measured arithmetic peak of this GPU's CUDA cores: the
// denominator of the evaluation kernels' roofline (the pair law runs on the
// FP32 or FP64 FMA pipes, not on tensor cores).
//
// Each thread advances kChains independent FMA chains for `iters` iterations
// (x <- x * a + b, never overflowing: |a| < 1), so the pipe, not a dependency,
// sets the rate.  Three forms: scalar FP32 FMA, packed FP32 (fma.rn.f32x2, two
// lanes per instruction, the form of the mixed evaluation) and FP64 DFMA.
// Timed with CUDA events on the caller's stream after one warm-up launch; no
// clock or other device setting is touched.  The paper derives its peaks from
// the hardware's unit counts and clock (Sect. 5.7, Table 2); this measures them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hg.h"
#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32(int iters, float a, float b, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[0] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32x2(int iters, float a, float b, float *sink)
{
    f2_t x[kChains];
    const f2_t a2 = f2_pack(a, a), b2 = f2_pack(b, b);
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = f2_pack((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = f2_fma(x[k], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        const float2 v = f2_unpack(x[k]);
        s += v.x + v.y;
    }
    if (s == 1234.5f) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f64(int iters, double a, double b, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5) sink[0] = s;
}

// One launch of `form` (0 f32, 1 f32x2, 2 f64) on `grid` CTAs.
cudaError_t launch_peak(int form, int grid, int iters, void *sink, cudaStream_t st)
{
    if (form == 0)
        k_peak_f32<<<grid, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-4f, static_cast<float *>(sink));
    else if (form == 1)
        k_peak_f32x2<<<grid, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-4f, static_cast<float *>(sink));
    else
        k_peak_f64<<<grid, kPeakThreads, 0, st>>>(iters, 0.999, 1e-4, static_cast<double *>(sink));
    return cudaGetLastError();
}

// Flops of one launch: grid * threads * iters * chains FMAs of 2 flops, per lane.
double peak_flops(int form, int grid, int iters)
{
    const double lanes = form == 1 ? 2.0 : 1.0;
    return 2.0 * lanes * (double)grid * kPeakThreads * (double)iters * kChains;
}

}  // namespace
}  // namespace hg

using namespace hg;

extern "C" int hg_peak_flops(int32_t form, int32_t device, void *stream, double *tflops, double *ms)
{
    set_call_error("");
    if (!tflops || form < 0 || form > 2) {
        set_call_error("form must be 0 (FP32 FMA), 1 (packed FP32 FMA) or 2 (FP64 FMA), tflops non-NULL");
        return HG_EINVAL;
    }
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        set_call_error("bad device");
        return HG_EINVAL;
    }
    int rc = HG_OK;
    int sms = 0, per_sm = 0;
    void *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The sink is never written (the chains never reach the test value), but it
    // must be a valid device address: the 8 bytes come from one small allocation.
    do {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess ||
            cudaMalloc(&sink, 16) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess) {
            set_call_error("device query, allocation or event creation failed");
            rc = HG_ECUDA;
            break;
        }
        const int grid = sms * (per_sm / kPeakThreads);   // every SM full
        const int iters = form == 2 ? 8192 : 262144;      // ~15-35 ms per launch
        if (launch_peak(form, grid, iters, sink, st) != cudaSuccess ||   // warm-up
            cudaEventRecord(e0, st) != cudaSuccess || launch_peak(form, grid, iters, sink, st) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            set_call_error("peak kernel failed");
            rc = HG_ECUDA;
            break;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || t <= 0.f) {
            set_call_error("event timing failed");
            rc = HG_ECUDA;
            break;
        }
        *tflops = peak_flops(form, grid, iters) / (1e-3 * t) / 1e12;
        if (ms) *ms = t;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaGetLastError();
    cudaSetDevice(prev);
    return rc;
}
