// hg_static.cu -- a stateless evaluation entry point that allocates no memory.
//
// Its scratch (packed j-records and the j-split partial sums) lives in one
// file-scope __device__ array of fixed size, so callers that are not allowed to
// allocate device memory can still run the evaluation kernel.  Every GPU that
// loads the library holds the array until the process exits.  All calls on a
// device share it: calls whose work overlaps on the GPU race with each other.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "hg.h"
#include "hg_internal.cuh"
#include "hg_kernels.cuh"

namespace hg {
namespace {

constexpr int64_t kStaticMaxN = 16384;                    // particles (multiple of the j-tiles)
constexpr size_t kRecBytes = 5 * (size_t)kStaticMaxN * 16;   // largest record layout (fp64: 80 B)
constexpr int64_t kStaticPcap = 4 * kStaticMaxN;            // partial sums: b * m <= kStaticPcap
constexpr size_t kPartBytes = (size_t)kStaticPcap * kOut * sizeof(double);
constexpr size_t kFlagBytes = 256;                          // int32 error word, int32 check flag
constexpr size_t kScratchBytes = kRecBytes + kPartBytes + kFlagBytes;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Slot {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of g_scratch on this device
    int sms = 0;
};
std::mutex g_mu;
Slot g_slots[kMaxDevices];

// Caller's predicted FP64 data -> j-records in the layout the evaluation reads
// (mixed: double-single positions and FP32 v, a, m; fp64: double2 pairs), with
// zero-mass padding up to npad.
template <bool MIXED>
__global__ void k_pack(int64_t n, int64_t npad, const double *mass, const double *x, const double *v,
                       const double *a, Records rec)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (MIXED) {
            MixedRecord r;
            if (i < n) {
                float hi[3], lo[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    hi[k] = __double2float_rn(x[3 * i + k]);
                    lo[k] = __double2float_rn(x[3 * i + k] - (double)hi[k]);
                }
                r = MixedRecord{hi[0], hi[1], hi[2], __double2float_rn(mass[i]), lo[0], lo[1], lo[2],
                                __double2float_rn(a[3 * i]), __double2float_rn(v[3 * i]),
                                __double2float_rn(v[3 * i + 1]), __double2float_rn(v[3 * i + 2]),
                                __double2float_rn(a[3 * i + 1]), __double2float_rn(a[3 * i + 2])};
            } else {
                const float far = (float)kPadCoord;
                r = MixedRecord{far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            }
            store_mixed_record(rec, i, r);
        } else {
            double2 q0, q1, q2, q3, q4;
            if (i < n) {
                q0 = make_double2(x[3 * i], x[3 * i + 1]);
                q1 = make_double2(x[3 * i + 2], mass[i]);
                q2 = make_double2(v[3 * i], v[3 * i + 1]);
                q3 = make_double2(v[3 * i + 2], a[3 * i]);
                q4 = make_double2(a[3 * i + 1], a[3 * i + 2]);
            } else {
                q0 = make_double2(kPadCoord, kPadCoord);
                q1 = make_double2(kPadCoord, 0.0);
                q2 = q3 = q4 = make_double2(0.0, 0.0);
            }
            static_cast<double2 *>(rec.p[0])[i] = q0;
            static_cast<double2 *>(rec.p[1])[i] = q1;
            static_cast<double2 *>(rec.p[2])[i] = q2;
            static_cast<double2 *>(rec.p[3])[i] = q3;
            static_cast<double2 *>(rec.p[4])[i] = q4;
        }
    }
}

// Device (or managed) memory that belongs to device `dev`, the current one: a
// pointer into another GPU's memory is refused, since the kernels would reach
// it without peer access.
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Once per device, with that device current: the device address of g_scratch
// (its host-side name is only a stand-in) and the kernel attributes.  Under
// CUDA's default lazy module loading this is also when the driver loads this
// file's module on the device and so allocates the array's memory.
int setup(int dev, Slot **out)
{
    if (dev < 0 || dev >= kMaxDevices) {
        set_call_error("device ordinal out of range for the static scratch");
        return HG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Slot &s = g_slots[dev];
    if (!s.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            set_call_error("cudaGetSymbolAddress of the static scratch failed");
            return HG_ECUDA;
        }
        if ((e = eval_setup(dev)) != cudaSuccess) {
            set_call_error("kernel attribute set-up failed");
            return HG_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            set_call_error("cudaDeviceGetAttribute failed");
            return HG_ECUDA;
        }
        s.base = static_cast<unsigned char *>(p);
        s.sms = sms;
        s.ready = true;
    }
    *out = &s;
    return HG_OK;
}

}  // namespace
}  // namespace hg

using namespace hg;

extern "C" int hg_evaluate_static(int64_t n, const double *mass, const double *pos, const double *vel,
                                  const double *acc_pred, double eps, int32_t precision, const int32_t *idx,
                                  int64_t m, double *acc, double *jerk, double *snap, void *stream)
{
    set_call_error("");
    if (n < 1 || n > kStaticMaxN) {
        set_call_error("n must be in [1, 16384]: the static scratch holds at most 16384 particles");
        return HG_EINVAL;
    }
    if (m < 0 || m > n) {
        set_call_error("m must be in [0, n]");
        return HG_EINVAL;
    }
    if (!(eps >= 0.0) || eps == INFINITY) {
        set_call_error("eps must be finite and >= 0");
        return HG_EINVAL;
    }
    if (precision != HG_FP64 && precision != HG_MIXED) {
        set_call_error("precision must be HG_FP64 or HG_MIXED");
        return HG_EINVAL;
    }
    if (!mass || !pos || !vel || !acc_pred || (m > 0 && (!idx || !acc || !jerk || !snap))) {
        set_call_error("every array argument is required");
        return HG_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_call_error("cudaGetDevice failed");
        return HG_ECUDA;
    }
    // The first call on a device loads the array (see setup); m = 0 does only that.
    Slot *slot = nullptr;
    int rc = setup(dev, &slot);
    if (rc || m == 0) return rc;
    const void *ptrs[] = {mass, pos, vel, acc_pred, idx, acc, jerk, snap};
    for (const void *q : ptrs)
        if (!on_device(q, dev)) {
            set_call_error("every array must be device memory of the current device");
            return HG_EINVAL;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool mixed = precision == HG_MIXED;
    unsigned char *base = slot->base;
    int32_t *err = reinterpret_cast<int32_t *>(base + kRecBytes + kPartBytes);
    int32_t *flag = err + 1;
    const int64_t npad = (n + kTJMixed - 1) / kTJMixed * kTJMixed;

    Records rec{};
    if (mixed) {   // six float4 arrays and one float2 array of npad / 2 record pairs
        for (int q = 0; q < kMixedArrays; ++q) rec.p[q] = base + q * (npad / 2) * 16;
    } else {
        for (int q = 0; q < 5; ++q) rec.p[q] = base + q * npad * 16;
    }
    // The array keeps the previous call's contents: clear the error word and flag.
    if (cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), st) != cudaSuccess ||
        launch_validate_idx(idx, m, n, flag, st) != cudaSuccess) {
        set_call_error("launch failed");
        return HG_ECUDA;
    }
    int32_t hflags[2] = {0, 0};
    if (cudaMemcpyAsync(hflags, err, sizeof(hflags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_call_error("index check failed");
        return HG_ECUDA;
    }
    if (hflags[1]) {
        set_call_error("idx must be strictly increasing and in [0, n)");
        return HG_EINVAL;
    }
    const int threads = 256;
    const int blocks = (int)((npad + threads - 1) / threads);
    if (mixed)
        k_pack<true><<<blocks, threads, 0, st>>>(n, npad, mass, pos, vel, acc_pred, rec);
    else
        k_pack<false><<<blocks, threads, 0, st>>>(n, npad, mass, pos, vel, acc_pred, rec);

    EvalArgs a{};           // every field zero unless set below (one system: bv.nc = 0)
    a.bv = BatchView{};
    a.rec = rec;
    a.npad = npad;
    a.n = n;
    a.pcap = kStaticPcap;
    a.idx = idx;
    a.m_dev = nullptr;
    a.m_host = m;
    a.plan_dev = nullptr;
    const PlanParams pq = plan_params(mixed, npad, slot->sms, kStaticPcap, 0, 0);
    a.plan_host = make_plan(m, pq);
    a.partial = reinterpret_cast<double *>(base + kRecBytes);
    a.eps2 = eps * eps;
    a.guard = eps * eps < kGuardEps2 ? 1 : 0;
    a.tx_extra = 0;
    a.err = err;
    a.direct_b1 = 0;        // partials summed by k_reduce
    if (cudaGetLastError() != cudaSuccess || launch_eval(mixed, a, slot->sms, st) != cudaSuccess ||
        launch_reduce(a, acc, jerk, snap, 2 * slot->sms, st) != cudaSuccess) {
        set_call_error("launch failed");
        return HG_ECUDA;
    }
    if (cudaMemcpyAsync(hflags, err, sizeof(hflags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_call_error("evaluation failed");
        return HG_ECUDA;
    }
    if (hflags[0] & ERR_TIMEOUT) {
        set_call_error("a bounded device wait expired");
        return HG_ETIMEOUT;
    }
    if (hflags[0] & ERR_BOUNDS) {
        set_call_error("a device bounds check failed (checked build)");
        return HG_ECUDA;
    }
    return HG_OK;
}
