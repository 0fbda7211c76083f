// hg_api.cu -- the C ABI of include/hg.h: context, device buffers, the
// explicit calls of one block step and the graph-captured device-resident
// stepping loop.
#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "hg.h"
#include "hg_internal.cuh"
#include "hg_kernels.cuh"

using namespace hg;

struct hg_ctx {
    int64_t n = 0, npad = 0;
    bool mixed = false;
    double eps = 0.0, eta = 0.0;
    hg_opts opts{};
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    State st{}, st2{};
    State own{};          // the context's own state arrays (st points at the caller's when bound)
    bool bound = false;
    Records rec{};
    int32_t *d_idx = nullptr, *d_idx2 = nullptr, *nb_cnt = nullptr, *nb_off = nullptr;
    double *nb_part = nullptr;
    DevScalars *d_sc = nullptr, *h_sc = nullptr;   // h_sc: pinned host mirror
    double *h_stage = nullptr;                     // pinned staging for small uploads
    int32_t *h_flags = nullptr;                    // pinned: (done, err) after two recent replays
    cudaEvent_t ev_flags[2] = {nullptr, nullptr};  // completion of those copies
    double *partial = nullptr;
    int64_t pcap = 0;
    PlanParams pp{};      // evaluation planner inputs
    BatchView bv{};       // independent clusters (bv.nc == 0: one system)
    std::vector<int64_t> cl_off_host;
    double *ra = nullptr, *rj = nullptr, *rs = nullptr;
    double *rn = nullptr;   // [n] noise scale of the evaluated particles (mixed)
    double *xe = nullptr, *ve = nullptr, *phi_part = nullptr, *e_part = nullptr, *e_out = nullptr;
    double *l_part = nullptr, *l_out = nullptr;   // angular momentum: 3 partials per CTA, result
    int e_splits = 0, e_g2 = 0;
    cudaGraphExec_t g_one = nullptr, g_many = nullptr;
    int64_t kernels = 0;            // kernel launches issued (graph replays count every node)
    std::vector<cudaEvent_t> ev_one, ev_many;   // profile: 6 events per captured block step
    double prof_ms[5] = {0, 0, 0, 0, 0};
    int64_t prof_steps = 0;
    bool tnext_valid = false;   // d_sc->tnext_bits = min_i tend_i of the current state
    double t_pred = NAN;    // time of the last hg_predict (NaN: none valid)
    int64_t cur_m = -1;     // size of the block from hg_next_block (-1: none)
    int64_t eval_m = -1;    // size of the last hg_evaluate (-1: none pending)
    double eval_t = NAN;
    std::vector<void *> dev_allocs;
    std::string err;
};

namespace {

thread_local std::string g_init_err;

// NVTX range named after the C ABI call for the duration of the call (a no-op
// unless a profiler is attached), e.g. ncu --nvtx --nvtx-include "hg_step/".
struct CallRange {
    explicit CallRange(const char *name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange &) = delete;
    CallRange &operator=(const CallRange &) = delete;
};

int fail(hg_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

// ---------------------------------------------------------------------------
// Host-side fault injection (testing): the nth device allocation or checked
// CUDA call after arming fails as if the CUDA runtime had refused it, without
// making the call.  Armed by hg_inject_fault or, at load, by the environment
// variable HG_FAULT=alloc:<n> or HG_FAULT=cuda:<n>.  Process-wide.
// ---------------------------------------------------------------------------
std::atomic<int32_t> g_fault_kind{HG_FAULT_NONE};
std::atomic<int64_t> g_fault_left{0};

// True for the armed fault point (which disarms the injector).
bool fault_point(int32_t kind)
{
    if (g_fault_kind.load(std::memory_order_relaxed) != kind) return false;
    if (g_fault_left.fetch_sub(1) != 1) return false;
    g_fault_kind.store(HG_FAULT_NONE);
    return true;
}

struct FaultFromEnv {
    FaultFromEnv()
    {
        const char *s = getenv("HG_FAULT");
        if (!s) return;
        const int32_t kind = strncmp(s, "alloc:", 6) == 0 ? HG_FAULT_ALLOC
                             : strncmp(s, "cuda:", 5) == 0 ? HG_FAULT_CUDA
                                                           : HG_FAULT_NONE;
        const long long nth = kind == HG_FAULT_NONE ? 0 : atoll(strchr(s, ':') + 1);
        if (nth > 0) {
            g_fault_left.store(nth);
            g_fault_kind.store(kind);
        }
    }
} g_fault_from_env;

constexpr cudaError_t kInjected = cudaErrorUnknown;

#define HG_CUDA(ctx, call)                                                                        \
    do {                                                                                          \
        const bool inj_ = fault_point(HG_FAULT_CUDA);                                             \
        cudaError_t e_ = inj_ ? kInjected : (call);                                               \
        if (e_ != cudaSuccess)                                                                    \
            return fail((ctx), HG_ECUDA,                                                          \
                        std::string(#call) + ": " + (inj_ ? "injected fault" : cudaGetErrorString(e_))); \
    } while (0)

bool is_pow2(double x)
{
    int e;
    return x > 0.0 && isfinite(x) && frexp(x, &e) == 0.5;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
T *dalloc(hg_ctx *c, int64_t count)
{
    void *p = nullptr;
    if (count < 1) count = 1;
    if (fault_point(HG_FAULT_ALLOC)) return nullptr;
    if (cudaMalloc(&p, (size_t)count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    c->dev_allocs.push_back(p);
    return static_cast<T *>(p);
}

bool alloc_state(hg_ctx *c, State &s)
{
    const int64_t n = c->n;
    s.mass = dalloc<double>(c, n);
    s.t = dalloc<double>(c, n);
    s.dt = dalloc<double>(c, n);
    s.tend = dalloc<double>(c, n);
    s.x = dalloc<double>(c, 3 * n);
    s.v = dalloc<double>(c, 3 * n);
    s.a = dalloc<double>(c, 3 * n);
    s.j = dalloc<double>(c, 3 * n);
    s.s = dalloc<double>(c, 3 * n);
    s.c = dalloc<double>(c, 3 * n);
    return s.mass && s.t && s.dt && s.tend && s.x && s.v && s.a && s.j && s.s && s.c;
}

StepParams step_params(const hg_ctx *c)
{
    StepParams p;
    p.eta = c->eta;
    p.eta_init = c->opts.eta_init;
    p.dt_min = c->opts.dt_min;
    p.dt_max = c->opts.dt_max;
    // FP32 pair terms carry ~3e-7 relative rounding, so the evaluated a_i errs
    // by up to ~3e-7 sum_j |a_ij|; a change below 3e-6 of the noise scale
    // sum_j m_j / r_ij^2 (>= sum_j |a_ij|) carries no usable higher-derivative
    // information.
    p.noise_rel = c->mixed ? 3e-6 : 0.0;
    p.log2_eta = (float)log2(c->eta);
    p.order = c->opts.order;
    return p;
}

EvalArgs eval_args(hg_ctx *c, const int64_t *m_dev, int64_t m_host)
{
    EvalArgs a;
    a.rec = c->rec;
    a.npad = c->npad;
    a.n = c->n;
    a.pcap = c->pcap;
    a.idx = c->d_idx;
    a.m_dev = m_dev;
    a.m_host = m_host;
    a.plan_dev = m_dev ? reinterpret_cast<const Plan *>(c->d_sc->plan) : nullptr;
    a.plan_host = m_dev ? Plan{} : make_plan(m_host, c->pp);
    a.partial = c->partial;
    a.eps2 = c->eps * c->eps;
    a.guard = c->eps * c->eps < kGuardEps2 ? 1 : 0;
    a.tx_extra = c->opts.test_stall_eval ? 16u : 0u;
    a.err = &c->d_sc->err;
    a.bv = c->bv;
    a.direct_b1 = c->bv.nc == 0 ? 1 : 0;   // one system: b = 1 plans write the results directly
    a.ra = c->ra;
    a.rj = c->rj;
    a.rs = c->rs;
    a.rn = c->mixed ? c->rn : nullptr;
    return a;
}

const int32_t *rmap_of(const hg_ctx *c) { return c->bv.nc > 0 ? c->bv.rmap : nullptr; }

// Work list over clusters; in graph steps it also counts the step's pair evaluations.
cudaError_t batch_plan(hg_ctx *c, const int64_t *m_dev, int64_t m_host, cudaStream_t s)
{
    return launch_batch_plan(c->d_idx, m_dev, m_host, c->bv, c->pp, m_dev ? c->d_sc : nullptr, s);
}

// Evaluation of the list in d_idx (host-known size m) into ra/rj/rs.
int run_eval_host_m(hg_ctx *c, int64_t m)
{
    EvalArgs a = eval_args(c, nullptr, m);
    if (c->bv.nc > 0) {
        HG_CUDA(c, batch_plan(c, nullptr, m, c->stream));
        c->kernels += 1;
    }
    HG_CUDA(c, launch_eval(c->mixed, a, c->num_sms, c->stream));
    HG_CUDA(c, launch_reduce(a, c->ra, c->rj, c->rs, 2 * c->num_sms, c->stream));
    c->kernels += 2;
    return HG_OK;
}

int sync_scalars(hg_ctx *c)
{
    HG_CUDA(c, cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->h_sc->err & ERR_TIMEOUT) return fail(c, HG_ETIMEOUT, "a bounded device wait expired");
    if (c->h_sc->err & ERR_BOUNDS)
        return fail(c, HG_ECUDA, "a device bounds check failed (checked build): an index, tile or partial-sum row "
                                 "was out of range and its access skipped");
    return HG_OK;
}

// Reset the validation flag, run a check, read it back.
template <class F>
int device_check(hg_ctx *c, F launch, int32_t *flag_out)
{
    HG_CUDA(c, cudaMemsetAsync(&c->d_sc->flag, 0, sizeof(int32_t), c->stream));
    HG_CUDA(c, launch(&c->d_sc->flag));
    c->kernels += 1;
    int rc = sync_scalars(c);
    if (rc) return rc;
    *flag_out = c->h_sc->flag;
    return HG_OK;
}

int upload_scalar(hg_ctx *c, double *dev_field, double v)
{
    HG_CUDA(c, cudaStreamSynchronize(c->stream));   // staging buffer is free
    c->h_stage[0] = v;
    HG_CUDA(c, cudaMemcpyAsync(dev_field, c->h_stage, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    return HG_OK;
}

// Kernels per graph-replayed block step: one system, selection + prediction,
// evaluation, reduction, correction (with the next minimum); clusters, three
// next-block passes, batch plan, prediction, evaluation, reduction, correction.
int step_kernels(const hg_ctx *c) { return c->bv.nc > 0 ? 8 : 4; }

// An event record that becomes a graph node when the stream is being captured
// (a plain record inside a capture only orders work and cannot be timed).
cudaError_t record_external(cudaEvent_t e, cudaStream_t s)
{
    return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
}

// One block step (Table 1 sections 1-4 and 8), sizes read on the device.
// ev: 6 events bracketing the 5 sections, or nullptr.
// One system: the selection is fused into the prediction (the "next" section
// is then empty) and the correction leaves the next block time, so a step is
// four kernels and starts from d_sc->tnext_bits.
int enqueue_block_step(hg_ctx *c, cudaStream_t s, const cudaEvent_t *ev)
{
    const bool batch = c->bv.nc > 0;
    if (ev) HG_CUDA(c, record_external(ev[0], s));
    if (batch) {
        HG_CUDA(c, launch_next_block(c->st, c->n, c->nb_part, c->nb_cnt, c->nb_off, c->d_idx, c->d_sc, 2, c->pp, s));
        HG_CUDA(c, batch_plan(c, &c->d_sc->m, 0, s));
    }
    if (ev) HG_CUDA(c, record_external(ev[1], s));
    if (batch)
        HG_CUDA(c, launch_predict_clusters(c->mixed, c->st, c->rec, c->n, c->bv, &c->d_sc->t_cur, &c->d_sc->m, s));
    else
        HG_CUDA(c, launch_predict_select(c->mixed, c->st, c->rec, c->n, c->npad, c->d_idx, c->d_sc, 1, c->pp,
                                         4 * c->num_sms, s));
    if (ev) HG_CUDA(c, record_external(ev[2], s));
    EvalArgs a = eval_args(c, &c->d_sc->m, 0);
    HG_CUDA(c, launch_eval(c->mixed, a, c->num_sms, s));
    if (ev) HG_CUDA(c, record_external(ev[3], s));
    HG_CUDA(c, launch_reduce(a, c->ra, c->rj, c->rs, 2 * c->num_sms, s));
    if (ev) HG_CUDA(c, record_external(ev[4], s));
    HG_CUDA(c, launch_correct(c->st, c->d_idx, &c->d_sc->m, 0, c->n, c->ra, c->rj, c->rs, a.rn, step_params(c),
                              c->d_sc, batch ? 0 : 1, 2 * c->num_sms, s));
    if (ev) HG_CUDA(c, record_external(ev[5], s));
    return HG_OK;
}

// A bound state (hg_bind_device) may have been written by the caller since the
// last call: rebuild what is derived from it (tend, the FP32 copies) before a
// call reads it.
int sync_bound(hg_ctx *c)
{
    if (!c->bound) return HG_OK;
    HG_CUDA(c, launch_tend(c->st, c->n, c->stream));
    c->kernels += 1;
    c->tnext_valid = false;
    return HG_OK;
}

// Graph steps of one system start from d_sc->tnext_bits: compute it when the
// state changed by other means (start-up, hg_set_state, hg_correct).
int ensure_tnext(hg_ctx *c)
{
    if (c->bv.nc > 0 || c->tnext_valid) return HG_OK;
    HG_CUDA(c, launch_next_min(c->st, c->n, c->nb_part, c->d_sc, c->stream));
    c->kernels += 1;
    c->tnext_valid = true;
    return HG_OK;
}

int capture(hg_ctx *c, int steps, cudaGraphExec_t *out, std::vector<cudaEvent_t> &ev)
{
    cudaGraph_t g = nullptr;
    if (c->opts.profile && ev.empty()) {
        ev.resize((size_t)steps * 6);
        for (auto &e : ev) HG_CUDA(c, cudaEventCreate(&e));
    }
    HG_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = HG_OK;
    for (int k = 0; k < steps && rc == HG_OK; ++k)
        rc = enqueue_block_step(c, c->cap_stream, c->opts.profile ? &ev[(size_t)k * 6] : nullptr);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc != HG_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(c, HG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, HG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return HG_OK;
}

int ensure_graphs(hg_ctx *c)
{
    int rc = HG_OK;
    if (!c->g_one) rc = capture(c, 1, &c->g_one, c->ev_one);
    if (rc == HG_OK && !c->g_many) rc = capture(c, c->opts.graph_steps, &c->g_many, c->ev_many);
    return rc;
}

// Launch one captured graph; with profiling, wait for it and add its section times.
int replay(hg_ctx *c, bool many)
{
    HG_CUDA(c, cudaGraphLaunch(many ? c->g_many : c->g_one, c->stream));
    const int steps = many ? c->opts.graph_steps : 1;
    c->kernels += (int64_t)step_kernels(c) * steps;
    if (!c->opts.profile) return HG_OK;
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    const std::vector<cudaEvent_t> &ev = many ? c->ev_many : c->ev_one;
    for (int k = 0; k < steps; ++k)
        for (int q = 0; q < 5; ++q) {
            float ms = 0.f;
            HG_CUDA(c, cudaEventElapsedTime(&ms, ev[(size_t)k * 6 + q], ev[(size_t)k * 6 + q + 1]));
            c->prof_ms[q] += ms;
        }
    c->prof_steps += steps;
    return HG_OK;
}

// Captured graphs hold kernel arguments by value (list pointers, planner
// inputs): drop them when those change; they are captured again on next use.
void drop_graphs(hg_ctx *c)
{
    if (c->g_one) {
        cudaGraphExecDestroy(c->g_one);
        c->g_one = nullptr;
    }
    if (c->g_many) {
        cudaGraphExecDestroy(c->g_many);
        c->g_many = nullptr;
    }
}

void invalidate(hg_ctx *c)
{
    c->t_pred = NAN;
    c->cur_m = -1;
    c->eval_m = -1;
    c->eval_t = NAN;
}

void release(hg_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->g_one) cudaGraphExecDestroy(c->g_one);
    if (c->g_many) cudaGraphExecDestroy(c->g_many);
    for (cudaEvent_t e : c->ev_one) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_many) cudaEventDestroy(e);
    for (void *p : c->dev_allocs) cudaFree(p);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    for (cudaEvent_t e : c->ev_flags)
        if (e) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

int init_impl(hg_ctx *c, const double *mass, const double *pos, const double *vel)
{
    const int64_t n = c->n;
    HG_CUDA(c, cudaSetDevice(c->device));
    cudaDeviceProp prop;
    HG_CUDA(c, cudaGetDeviceProperties(&prop, c->device));
    c->num_sms = prop.multiProcessorCount;
    if (c->opts.stream) {
        c->stream = static_cast<cudaStream_t>(c->opts.stream);
    } else {
        HG_CUDA(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    HG_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    HG_CUDA(c, cudaMallocHost(reinterpret_cast<void **>(&c->h_sc), sizeof(DevScalars)));
    HG_CUDA(c, cudaMallocHost(reinterpret_cast<void **>(&c->h_stage), 4 * sizeof(double)));
    HG_CUDA(c, cudaMallocHost(reinterpret_cast<void **>(&c->h_flags), 4 * sizeof(int32_t)));
    for (cudaEvent_t &e : c->ev_flags) HG_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

    const int64_t tj = kTJMixed > kTJF64 ? kTJMixed : kTJF64;
    c->npad = (n + tj - 1) / tj * tj;
    // Clusters: each cluster's records start on a tile boundary of both layouts.
    const int nc = c->cl_off_host.empty() ? 0 : (int)c->cl_off_host.size() - 1;
    std::vector<int64_t> rec_off;
    std::vector<int32_t> rmap, cl_of;
    int64_t pcap_clusters = 0;
    if (nc > 0) {
        rec_off.assign((size_t)nc + 1, 0);
        rmap.resize((size_t)n);
        cl_of.resize((size_t)n);
        for (int k = 0; k < nc; ++k) {
            const int64_t a = c->cl_off_host[k], b = c->cl_off_host[k + 1];
            rec_off[k + 1] = rec_off[k] + (b - a + tj - 1) / tj * tj;
            for (int64_t i = a; i < b; ++i) {
                rmap[(size_t)i] = (int32_t)(rec_off[k] + (i - a));
                cl_of[(size_t)i] = k;
            }
            const int64_t ntc = (rec_off[k + 1] - rec_off[k]) / (c->mixed ? kTJMixed : kTJF64);
            pcap_clusters += (ntc + kBatchTpsMax - 1) / kBatchTpsMax * (b - a);
        }
        c->npad = rec_off[(size_t)nc];
        if (c->npad > (int64_t)INT32_MAX) return fail(c, HG_EINVAL, "too many padded records");
    }
    bool ok = alloc_state(c, c->st) && alloc_state(c, c->st2);
    if (c->mixed) {   // the FP32 copies read by the mixed predictor (4 float4 per particle)
        c->st.f32 = dalloc<float4>(c, 4 * n);
        ok = ok && c->st.f32;
    }
    c->own = c->st;
    if (c->mixed) {
        for (int q = 0; q < kMixedArrays; ++q) {   // record pairs: six float4 arrays and one float2
            c->rec.p[q] = q < 6 ? (void *)dalloc<float4>(c, c->npad / 2) : (void *)dalloc<float2>(c, c->npad / 2);
            ok = ok && c->rec.p[q];
        }
    } else {
        for (int q = 0; q < 5; ++q) {
            c->rec.p[q] = dalloc<double2>(c, c->npad);
            ok = ok && c->rec.p[q];
        }
    }
    c->d_idx = dalloc<int32_t>(c, n);
    c->d_idx2 = dalloc<int32_t>(c, n);
    const int g = nb_grid(n);
    c->nb_part = dalloc<double>(c, g);
    c->nb_cnt = dalloc<int32_t>(c, g);
    c->nb_off = dalloc<int32_t>(c, g);
    c->d_sc = dalloc<DevScalars>(c, 1);
    // Partial sums: b * m <= pcap (b never exceeds the number of j-tiles).
    const int64_t max_tiles = c->npad / (c->mixed ? kTJMixed : kTJF64);
    int64_t pcap = 4 * n > (1 << 20) ? 4 * n : (1 << 20);
    if (pcap > max_tiles * n) pcap = max_tiles * n;
    if (nc > 0) pcap = 4 * n + pcap_clusters;   // the coarsest batch split always fits
    c->pcap = pcap;
    if (nc > 0) {
        BatchView &bv = c->bv;
        bv.nc = nc;
        int64_t *clo = dalloc<int64_t>(c, nc + 1), *ro = dalloc<int64_t>(c, nc + 1);
        int32_t *rm = dalloc<int32_t>(c, n), *co = dalloc<int32_t>(c, n);
        bv.a_off = dalloc<int64_t>(c, nc + 1);
        bv.item_off = dalloc<int64_t>(c, nc + 1);
        bv.part_off = dalloc<int64_t>(c, nc + 1);
        bv.pred_off = dalloc<int64_t>(c, nc + 1);
        bv.tpi_c = dalloc<int32_t>(c, nc);
        bv.b_c = dalloc<int32_t>(c, nc);
        bv.tps = dalloc<int64_t>(c, 1);
        if (!clo || !ro || !rm || !co || !bv.a_off || !bv.item_off || !bv.part_off || !bv.pred_off || !bv.tpi_c ||
            !bv.b_c || !bv.tps)
            return fail(c, HG_ENOMEM, "device allocation failed");
        HG_CUDA(c, cudaMemcpy(clo, c->cl_off_host.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        HG_CUDA(c, cudaMemcpy(ro, rec_off.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        HG_CUDA(c, cudaMemcpy(rm, rmap.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        HG_CUDA(c, cudaMemcpy(co, cl_of.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        bv.cl_off = clo;
        bv.rec_off = ro;
        bv.rmap = rm;
        bv.cl_of = co;
    }
    c->partial = dalloc<double>(c, (int64_t)kOut * pcap);
    c->ra = dalloc<double>(c, 3 * n);
    c->rj = dalloc<double>(c, 3 * n);
    c->rs = dalloc<double>(c, 3 * n);
    c->rn = dalloc<double>(c, n);
    c->xe = dalloc<double>(c, 3 * n);
    c->ve = dalloc<double>(c, 3 * n);
    c->e_splits = energy_splits(n, c->num_sms);
    c->phi_part = dalloc<double>(c, (int64_t)c->e_splits * n);
    c->e_g2 = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    c->e_part = dalloc<double>(c, 2 * c->e_g2);
    c->e_out = dalloc<double>(c, 2);
    c->l_part = dalloc<double>(c, 3 * c->e_g2);
    c->l_out = dalloc<double>(c, 3);
    ok = ok && c->d_idx && c->d_idx2 && c->nb_part && c->nb_cnt && c->nb_off && c->d_sc && c->partial && c->ra &&
         c->rj && c->rs && c->rn && c->xe && c->ve && c->phi_part && c->e_part && c->e_out && c->l_part && c->l_out;
    if (!ok) return fail(c, HG_ENOMEM, "device allocation failed");

    HG_CUDA(c, eval_setup(c->device));
    c->pp = plan_params(c->mixed, c->npad, c->num_sms, c->pcap, c->opts.tpi, c->opts.jsplit);
    if (nc > 0) c->pp.variants = 1;   // the cluster work list is built for the first kernel variant

    DevScalars z{};
    z.t_stop = INFINITY;
    *c->h_sc = z;
    HG_CUDA(c, cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream));
    HG_CUDA(c, cudaMemcpyAsync(c->st.mass, mass, n * sizeof(double), cudaMemcpyDefault, c->stream));
    HG_CUDA(c, cudaMemcpyAsync(c->st.x, pos, 3 * n * sizeof(double), cudaMemcpyDefault, c->stream));
    HG_CUDA(c, cudaMemcpyAsync(c->st.v, vel, 3 * n * sizeof(double), cudaMemcpyDefault, c->stream));
    int32_t flag = 0;
    int rc = device_check(
        c,
        [&](int32_t *f) {
            return launch_validate_init(c->st.mass, c->st.x, c->st.v, n, value_limits(c->mixed, c->eps), f, c->stream);
        },
        &flag);
    if (rc) return rc;
    if (flag)
        return fail(c, HG_EINVAL,
                    c->mixed ? "masses must be finite, > 0 and <= 1e37 min(1, eps^3), |positions| <= 1e15 and "
                               "|velocities| <= 1e30 (the FP32 range of the mixed pair arithmetic)"
                             : "masses must be finite, > 0 and <= 1e300 min(1, eps^3), |positions| and |velocities| "
                               "<= 1e150");

    // Start-up: every particle active at t = 0; the prediction is the identity.
    for (double *p : {c->st.a, c->st.j, c->st.s, c->st.c})
        HG_CUDA(c, cudaMemsetAsync(p, 0, 3 * n * sizeof(double), c->stream));
    HG_CUDA(c, cudaMemsetAsync(c->st.t, 0, n * sizeof(double), c->stream));
    if (c->opts.start_mode == 1) {
        std::vector<double> dtv((size_t)n, c->opts.dt_max);
        HG_CUDA(c, cudaMemcpyAsync(c->st.dt, dtv.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        HG_CUDA(c, launch_tend(c->st, n, c->stream));
        rc = sync_scalars(c);
        if (rc) return rc;
        invalidate(c);
        return HG_OK;
    }
    std::vector<int32_t> iota((size_t)n);
    for (int64_t i = 0; i < n; ++i) iota[(size_t)i] = (int32_t)i;
    HG_CUDA(c, cudaMemcpyAsync(c->d_idx, iota.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    if (c->bv.nc > 0) HG_CUDA(c, launch_pad_records(c->mixed, c->rec, c->npad, c->stream));
    HG_CUDA(c, launch_f32(c->st, n, c->stream));
    HG_CUDA(c, launch_predict(c->mixed, c->st, c->rec, n, c->npad, nullptr, 0.0, nullptr, rmap_of(c), c->stream));
    rc = run_eval_host_m(c, n);
    if (rc) return rc;
    HG_CUDA(c, launch_start(c->st, n, c->ra, c->rj, c->rs, step_params(c), c->stream));
    HG_CUDA(c, launch_f32(c->st, n, c->stream));
    rc = sync_scalars(c);
    if (rc) return rc;
    invalidate(c);
    return HG_OK;
}

// ---------------------------------------------------------------------------
// Autotuning of the evaluation plan per block-size bucket.
// ---------------------------------------------------------------------------
constexpr int kTuneCand = 14;        // cheapest plans of the cost model timed per bucket
constexpr double kTuneGain = 0.97;   // a rival is stored only if at least 3% faster
constexpr double kTuneTargetUs = 2000.0;

// Mean device time of `reps` evaluations + reductions of the list in d_idx with
// the current planner inputs, after one warm-up (reps == 0: chosen from the
// warm-up's time so that the timed launches take ~2 ms, 3..64).
int time_eval(hg_ctx *c, int64_t m, int *reps, cudaEvent_t e0, cudaEvent_t e1, double *us)
{
    HG_CUDA(c, cudaEventRecord(e0, c->stream));
    int rc = run_eval_host_m(c, m);
    if (rc) return rc;
    HG_CUDA(c, cudaEventRecord(e1, c->stream));
    HG_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    HG_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    if (*reps <= 0) {
        const double one = ms > 0.f ? 1000.0 * ms : 1.0;
        *reps = (int)std::min(64.0, std::max(3.0, ceil(kTuneTargetUs / one)));
    }
    HG_CUDA(c, cudaEventRecord(e0, c->stream));
    for (int r = 0; r < *reps; ++r)
        if ((rc = run_eval_host_m(c, m)) != HG_OK) return rc;
    HG_CUDA(c, cudaEventRecord(e1, c->stream));
    HG_CUDA(c, cudaEventSynchronize(e1));
    HG_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    *us = 1000.0 * ms / *reps;
    return HG_OK;
}

// Table values to time for a block of m: the cost model's choice first, then
// its cheapest rivals (one system: distinct (tpi, b) plans, cheapest first, plus
// the cheapest of every tpi; clusters: every batch code).
std::vector<int> tune_candidates(const hg_ctx *c, int64_t m)
{
    std::vector<int> out;
    if (c->bv.nc > 0) {
        out.push_back(1 + 8 * 1);   // the untuned knobs w = 1, s = 0
        for (int s = 0; s <= 2; ++s)
            for (int w = 0; w <= kBatchWMax; ++w)
                if (w + 8 * s != out[0]) out.push_back(w + 8 * s);
        return out;
    }
    PlanParams q = c->pp;
    for (int k = 0; k < kTuneBuckets; ++k) q.tuned[k] = -1;
    struct Cand {
        int64_t cost;
        int c, tpi, b, v;
    };
    std::vector<Cand> all;
    for (int k = 0; k < plan_total(q); ++k) {
        Plan p;
        const int64_t cost = plan_candidate(m, q, k, p);
        if (cost < 0) continue;
        bool dup = false;
        for (const Cand &x : all) dup = dup || (x.tpi == p.tpi && x.b == p.b && x.v == p.variant);
        if (!dup) all.push_back(Cand{cost, k, p.tpi, p.b, p.variant});
    }
    std::stable_sort(all.begin(), all.end(), [](const Cand &a, const Cand &b) { return a.cost < b.cost; });
    std::vector<bool> take(all.size(), false);
    for (size_t k = 0; k < all.size() && (int)k < kTuneCand; ++k) take[k] = true;
    for (int v = 0; v < q.variants; ++v)
        for (int t = 1; t <= kMaxTPI; t *= 2)
            for (size_t k = 0; k < all.size(); ++k)
                if (all[k].tpi == t && all[k].v == v) {
                    take[k] = true;
                    break;
                }
    for (size_t k = 0; k < all.size(); ++k)
        if (take[k]) out.push_back(all[k].c);
    return out;
}

int tune_impl(hg_ctx *c, int64_t m_max, int32_t reps_in, hg_tune_entry *report, int32_t cap, int32_t *n_out)
{
    const int64_t n = c->n;
    if (m_max <= 0) {   // automatic: evaluations of up to ~2^32 (mixed) or 2^28 (FP64) pair interactions
        const int64_t budget = c->mixed ? ((int64_t)1 << 32) : ((int64_t)1 << 28);
        m_max = std::max<int64_t>(1, budget / n);
    }
    const int64_t mtop = std::min(m_max, n);
    // Representative blocks: the particles with the smallest steps are the ones
    // the block scheme makes active most often.
    std::vector<double> dt((size_t)n);
    HG_CUDA(c, cudaMemcpyAsync(dt.data(), c->st.dt, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<int32_t> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return dt[(size_t)a] < dt[(size_t)b]; });
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HG_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, HG_ECUDA, "cudaEventCreate failed");
    }
    drop_graphs(c);
    invalidate(c);
    int rc = HG_OK;
    int32_t count = 0;
    std::vector<int32_t> list;
    for (int k = 0; k <= tune_bucket(mtop) && rc == HG_OK; ++k) {
        // Timed at block sizes spread over the bucket (tune_points); the
        // reported m is the bucket's middle one.
        const int64_t m = k == 0 ? 1 : std::min<int64_t>(mtop, (int64_t)3 << (k - 1));
        int64_t pts_a[3];
        const std::vector<int64_t> pts(pts_a, pts_a + tune_points(k, mtop, pts_a));
        const std::vector<int> cand = tune_candidates(c, m);
        std::vector<double> sum(cand.size(), 0.0);
        for (size_t pi = 0; pi < pts.size() && rc == HG_OK; ++pi) {
            const int64_t mp = pts[pi];
            list.assign(order.begin(), order.begin() + mp);
            std::sort(list.begin(), list.end());
            if (cudaMemcpyAsync(c->d_idx, list.data(), mp * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess) {
                rc = fail(c, HG_ECUDA, "list upload failed");
                break;
            }
            int reps = reps_in;
            for (size_t q = 0; q < cand.size() && rc == HG_OK; ++q) {
                c->pp.tuned[k] = q == 0 ? -1 : (int16_t)cand[q];   // q == 0: the cost model itself
                double us = 0.0;
                rc = time_eval(c, mp, &reps, e0, e1, &us);
                sum[q] += us;
            }
        }
        if (rc) break;
        size_t best = 0;
        for (size_t q = 1; q < cand.size(); ++q)
            if (sum[q] < sum[best]) best = q;
        const int chosen = (best > 0 && sum[best] < kTuneGain * sum[0]) ? cand[best] : -1;
        c->pp.tuned[k] = (int16_t)chosen;
        if (report && count < cap) {
            hg_tune_entry &e = report[count];
            e.m = m;
            e.bucket = k;
            e.candidates = (int32_t)cand.size();
            e.model = cand[0];
            e.chosen = chosen;
            e.model_us = sum[0] / (double)pts.size();
            e.best_us = chosen >= 0 ? sum[best] / (double)pts.size() : e.model_us;
        }
        ++count;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (n_out) *n_out = count;
    return sync_scalars(c);
}

}  // namespace

void hg::set_call_error(const char *msg) { g_init_err = msg; }

extern "C" {

void hg_default_opts(hg_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = HG_FP64;
    o->energy_precision = HG_FP64;
    o->device = 0;
    o->tpi = 0;
    o->jsplit = 0;
    o->graph_steps = 8;
    o->start_mode = 0;
    o->profile = 0;
    o->test_stall_eval = 0;
    o->order = 6;
    o->dt_min = 1.0 / 33554432.0;   // 2^-25
    o->dt_max = 0.125;              // 2^-3
    o->eta_init = 0.01;
    o->stream = nullptr;
}

const char *hg_init_error(void) { return g_init_err.c_str(); }

int hg_init(hg_ctx **out, int64_t n, const double *mass, const double *pos, const double *vel, double eps,
            double eta, const hg_opts *opts)
{
    return hg_init_batch(out, 0, nullptr, n, mass, pos, vel, eps, eta, opts);
}

int hg_init_batch(hg_ctx **out, int32_t n_clusters, const int64_t *offsets, int64_t n, const double *mass,
                  const double *pos, const double *vel, double eps, double eta, const hg_opts *opts)
{
    const CallRange range_("hg_init_batch");
    g_init_err.clear();
    auto bad = [](const char *m) {
        g_init_err = m;
        return HG_EINVAL;
    };
    if (!out) return bad("out is NULL");
    *out = nullptr;
    if (n < 1 || n > (int64_t)INT32_MAX - 1024) return bad("n must be in [1, 2^31 - 1025]");
    std::vector<int64_t> cl;
    if (n_clusters < 0) return bad("n_clusters must be >= 0");
    if (n_clusters > 0) {
        if (!offsets) return bad("offsets are required with clusters");
        cl.resize((size_t)n_clusters + 1);
        if (cudaMemcpy(cl.data(), offsets, cl.size() * sizeof(int64_t), cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return bad("offsets could not be read");
        }
        if (cl[0] != 0 || cl[(size_t)n_clusters] != n) return bad("offsets must start at 0 and end at n");
        for (int32_t k = 0; k < n_clusters; ++k)
            if (cl[(size_t)k + 1] <= cl[(size_t)k]) return bad("every cluster needs at least one particle");
    }
    if (!mass || !pos || !vel) return bad("mass, pos and vel are required");
    if (!isfinite(eps) || eps < 0.0) return bad("eps must be finite and >= 0");
    if (!isfinite(eta) || eta <= 0.0) return bad("eta must be finite and > 0");
    hg_opts o;
    if (opts)
        o = *opts;
    else
        hg_default_opts(&o);
    if (o.precision != HG_FP64 && o.precision != HG_MIXED) return bad("precision must be HG_FP64 or HG_MIXED");
    if (eps > value_limits(o.precision == HG_MIXED, eps).pos)
        return bad("eps must not exceed the position limit (mixed 1e15, FP64 1e150)");
    if (o.energy_precision != HG_FP64 && o.energy_precision != HG_MIXED) return bad("bad energy_precision");
    if (!is_pow2(o.dt_min) || !is_pow2(o.dt_max) || o.dt_min > o.dt_max)
        return bad("dt_min and dt_max must be powers of two with dt_min <= dt_max");
    if (!isfinite(o.eta_init) || o.eta_init <= 0.0) return bad("eta_init must be finite and > 0");
    if (o.tpi != 0 && (o.tpi < 0 || o.tpi > kMaxTPI || (o.tpi & (o.tpi - 1)) != 0))
        return bad("tpi must be 0 or a power of two <= 64");
    if (o.jsplit < 0) return bad("jsplit must be >= 0");
    if (o.graph_steps < 1 || o.graph_steps > 1024) return bad("graph_steps must be in [1, 1024]");
    if (o.start_mode != 0 && o.start_mode != 1) return bad("start_mode must be 0 or 1");
    if (o.test_stall_eval != 0 && o.test_stall_eval != 1) return bad("test_stall_eval must be 0 or 1");
    if (o.order == 0) o.order = 6;
    if (o.order != 4 && o.order != 6) return bad("order must be 4 or 6");

    hg_ctx *c = new (std::nothrow) hg_ctx();
    if (!c) {
        g_init_err = "host allocation failed";
        return HG_ENOMEM;
    }
    c->n = n;
    c->mixed = o.precision == HG_MIXED;
    c->eps = eps;
    c->eta = eta;
    c->opts = o;
    c->device = o.device;
    c->cl_off_host = std::move(cl);
    int rc = init_impl(c, mass, pos, vel);
    if (rc != HG_OK) {
        g_init_err = c->err;
        release(c);
        return rc;
    }
    *out = c;
    return HG_OK;
}

int hg_next_block(hg_ctx *c, double *t_next, int32_t *idx, int64_t cap, int64_t *m_out)
{
    const CallRange range_("hg_next_block");
    if (!c) return HG_EINVAL;
    if (const int rb = sync_bound(c)) return rb;
    HG_CUDA(c, launch_next_block(c->st, c->n, c->nb_part, c->nb_cnt, c->nb_off, c->d_idx, c->d_sc, 0, c->pp,
                                 c->stream));
    c->kernels += 3;
    int rc = sync_scalars(c);
    if (rc) return rc;
    const int64_t m = c->h_sc->m;
    invalidate(c);
    c->cur_m = m;
    if (t_next) *t_next = c->h_sc->t_cur;
    if (m_out) *m_out = m;
    if (idx) {
        if (cap < m) return fail(c, HG_EINVAL, "idx capacity smaller than the block");
        HG_CUDA(c, cudaMemcpyAsync(idx, c->d_idx, m * sizeof(int32_t), cudaMemcpyDefault, c->stream));
        HG_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return HG_OK;
}

int hg_predict(hg_ctx *c, double t)
{
    const CallRange range_("hg_predict");
    if (!c) return HG_EINVAL;
    if (!isfinite(t)) return fail(c, HG_EINVAL, "t must be finite");
    if (const int rb = sync_bound(c)) return rb;
    HG_CUDA(c, launch_predict(c->mixed, c->st, c->rec, c->n, c->npad, nullptr, t, nullptr, rmap_of(c), c->stream));
    c->kernels += 1;
    c->t_pred = t;
    c->eval_m = -1;
    return HG_OK;
}

int hg_evaluate(hg_ctx *c, const int32_t *idx, int64_t m, double *acc, double *jerk, double *snap)
{
    const CallRange range_("hg_evaluate");
    if (!c) return HG_EINVAL;
    if (isnan(c->t_pred)) return fail(c, HG_ESTATE, "hg_evaluate needs a preceding hg_predict");
    if (m < 0 || m > c->n) return fail(c, HG_EINVAL, "m must be in [0, n]");
    if (!idx) {
        if (c->cur_m < 0 || m != c->cur_m) return fail(c, HG_EINVAL, "idx NULL needs m equal to the current block");
    } else if (m > 0) {
        if (is_device_ptr(idx)) {
            HG_CUDA(c, cudaMemcpyAsync(c->d_idx2, idx, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
            int32_t flag = 0;
            int rc = device_check(
                c, [&](int32_t *f) { return launch_validate_idx(c->d_idx2, m, c->n, f, c->stream); }, &flag);
            if (rc) return rc;
            if (flag) return fail(c, HG_EINVAL, "idx must be strictly increasing and in [0, n)");
        } else {
            for (int64_t q = 0; q < m; ++q)
                if (idx[q] < 0 || idx[q] >= c->n || (q > 0 && idx[q] <= idx[q - 1]))
                    return fail(c, HG_EINVAL, "idx must be strictly increasing and in [0, n)");
            HG_CUDA(c, cudaMemcpyAsync(c->d_idx2, idx, m * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        }
        int32_t *t = c->d_idx;
        c->d_idx = c->d_idx2;
        c->d_idx2 = t;
        c->cur_m = m;
        drop_graphs(c);   // they captured the old list pointer
    }
    if (m > 0) {
        int rc = run_eval_host_m(c, m);
        if (rc) return rc;
        double *outs[3] = {acc, jerk, snap};
        const double *res[3] = {c->ra, c->rj, c->rs};
        for (int k = 0; k < 3; ++k)
            if (outs[k])
                HG_CUDA(c, cudaMemcpyAsync(outs[k], res[k], 3 * m * sizeof(double), cudaMemcpyDefault, c->stream));
    }
    int rc = sync_scalars(c);
    if (rc) return rc;
    c->eval_m = m;
    c->eval_t = c->t_pred;
    return HG_OK;
}

int hg_condition_scale(hg_ctx *c, double *out, int64_t m)
{
    const CallRange range_("hg_condition_scale");
    if (!c) return HG_EINVAL;
    if (!c->mixed) return fail(c, HG_ESTATE, "the FP64 evaluation does not form the condition scale");
    if (c->eval_m < 0) return fail(c, HG_ESTATE, "hg_condition_scale needs a preceding hg_evaluate");
    if (m != c->eval_m || (m > 0 && !out)) return fail(c, HG_EINVAL, "m differs from the last hg_evaluate");
    if (m > 0) HG_CUDA(c, cudaMemcpyAsync(out, c->rn, m * sizeof(double), cudaMemcpyDefault, c->stream));
    return sync_scalars(c);
}

int hg_correct(hg_ctx *c, const int32_t *idx, int64_t m)
{
    const CallRange range_("hg_correct");
    if (!c) return HG_EINVAL;
    if (c->eval_m < 0) return fail(c, HG_ESTATE, "hg_correct needs a preceding hg_evaluate");
    if (m != c->eval_m) return fail(c, HG_EINVAL, "m differs from the last hg_evaluate");
    if (m == 0) {
        c->eval_m = -1;
        return HG_OK;
    }
    const int32_t *given = nullptr;
    if (idx) {
        HG_CUDA(c, cudaMemcpyAsync(c->d_idx2, idx, m * sizeof(int32_t), cudaMemcpyDefault, c->stream));
        given = c->d_idx2;
    }
    int32_t flag = 0;
    int rc = device_check(
        c, [&](int32_t *f) { return launch_check_correct(c->st, given, c->d_idx, m, c->n, c->eval_t, f, c->stream); },
        &flag);
    if (rc) return rc;
    if (flag)
        return fail(c, HG_ESTATE, "list differs from the evaluation, or a particle is not due at the block time");
    // 3 lanes per particle, units of 10 particles per warp, 4 warps per CTA
    const int cgrid = (int)std::min<int64_t>(((m + 9) / 10 + 3) / 4, 2 * (int64_t)c->num_sms);
    HG_CUDA(c, launch_correct(c->st, c->d_idx, nullptr, m, c->n, c->ra, c->rj, c->rs, c->mixed ? c->rn : nullptr,
                              step_params(c), c->d_sc, 0, cgrid, c->stream));
    c->tnext_valid = false;
    c->kernels += 1;
    rc = upload_scalar(c, &c->d_sc->t_cur, c->eval_t);
    if (rc) return rc;
    invalidate(c);
    return HG_OK;
}

int hg_step(hg_ctx *c, int64_t n_steps)
{
    const CallRange range_("hg_step");
    if (!c) return HG_EINVAL;
    if (n_steps < 0) return fail(c, HG_EINVAL, "n_steps must be >= 0");
    if (n_steps == 0) return HG_OK;
    int rc = sync_bound(c);
    if (rc == HG_OK) rc = ensure_graphs(c);
    if (rc == HG_OK) rc = ensure_tnext(c);
    if (rc) return rc;
    invalidate(c);
    const int64_t s = c->opts.graph_steps;
    for (int64_t k = 0; k < n_steps / s; ++k)
        if ((rc = replay(c, true)) != HG_OK) return rc;
    for (int64_t k = 0; k < n_steps % s; ++k)
        if ((rc = replay(c, false)) != HG_OK) return rc;
    return HG_OK;
}

int hg_advance(hg_ctx *c, double t_end, int64_t *steps_out)
{
    const CallRange range_("hg_advance");
    if (!c) return HG_EINVAL;
    if (!isfinite(t_end)) return fail(c, HG_EINVAL, "t_end must be finite");
    int rc = sync_bound(c);
    if (rc == HG_OK) rc = ensure_graphs(c);
    if (rc == HG_OK) rc = ensure_tnext(c);
    if (rc) return rc;
    invalidate(c);
    rc = sync_scalars(c);
    if (rc) return rc;
    const int64_t steps0 = c->h_sc->steps;
    rc = upload_scalar(c, &c->d_sc->t_stop, t_end);
    if (rc) return rc;
    HG_CUDA(c, cudaMemsetAsync(&c->d_sc->done, 0, sizeof(int32_t), c->stream));
    if (c->opts.profile) {   // profiled replays synchronise anyway: check after each
        for (;;) {
            rc = replay(c, true);
            if (rc) break;
            rc = sync_scalars(c);
            if (rc) break;
            if (c->h_sc->done) break;
        }
    } else {
        // Keep the next replay queued while the flags of the previous one are
        // read, so that the GPU never waits for the host.  Replays past the
        // stop time are empty block steps (m = 0, every kernel returns at
        // once): at most one such graph runs per call.
        static_assert(offsetof(DevScalars, err) == offsetof(DevScalars, done) + sizeof(int32_t),
                      "done and err are adjacent");
        // A failed CUDA call ends the loop with its status (not a return), so
        // that the stop time is reset and the stream drained below.
        auto cuda_rc = [&](cudaError_t e, const char *what) {
            return e == cudaSuccess ? HG_OK : fail(c, HG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
        };
        for (int64_t k = 0;; ++k) {
            const int slot = (int)(k & 1);
            if ((rc = replay(c, true)) != HG_OK) break;
            int32_t *flags = c->h_flags + 2 * slot;
            rc = cuda_rc(cudaMemcpyAsync(flags, &c->d_sc->done, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                         c->stream),
                         "flag copy");
            if (rc == HG_OK) rc = cuda_rc(cudaEventRecord(c->ev_flags[slot], c->stream), "flag event");
            if (rc) break;
            if (k == 0) continue;
            const int prev = slot ^ 1;
            if ((rc = cuda_rc(cudaEventSynchronize(c->ev_flags[prev]), "flag wait")) != HG_OK) break;
            const int32_t *pf = c->h_flags + 2 * prev;
            if (pf[1] & ERR_TIMEOUT) break;   // reported by the final read below
            if (pf[0]) break;
        }
        const int rs = sync_scalars(c);   // waits for the queued replay whatever happened
        if (rc == HG_OK) rc = rs;
    }
    int rc2 = upload_scalar(c, &c->d_sc->t_stop, INFINITY);
    if (rc) return rc;
    if (rc2) return rc2;
    if (steps_out) *steps_out = c->h_sc->steps - steps0;
    return HG_OK;
}

int hg_energy(hg_ctx *c, double *kinetic, double *potential)
{
    const CallRange range_("hg_energy");
    if (!c) return HG_EINVAL;
    int rc = sync_scalars(c);
    if (rc) return rc;
    const double t = c->h_sc->t_cur;
    c->kernels += 4;
    HG_CUDA(c, launch_energy(c->opts.energy_precision == HG_MIXED, c->st, c->n, t, c->eps * c->eps, c->xe, c->ve,
                             c->phi_part, c->e_splits, c->e_part, c->e_g2, c->e_out, c->bv, c->stream));
    HG_CUDA(c, cudaMemcpyAsync(c->h_stage, c->e_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (kinetic) *kinetic = c->h_stage[0];
    if (potential) *potential = c->h_stage[1];
    return HG_OK;
}

int hg_angular_momentum(hg_ctx *c, double *L)
{
    const CallRange range_("hg_angular_momentum");
    if (!c || !L) return HG_EINVAL;
    int rc = sync_scalars(c);
    if (rc) return rc;
    c->kernels += 3;
    HG_CUDA(c, launch_angular_momentum(c->st, c->n, c->h_sc->t_cur, c->xe, c->ve, c->l_part, c->e_g2, c->l_out,
                                       c->stream));
    HG_CUDA(c, cudaMemcpyAsync(c->h_stage, c->l_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; ++k) L[k] = c->h_stage[k];
    return HG_OK;
}

int hg_get_state(hg_ctx *c, hg_state *o)
{
    const CallRange range_("hg_get_state");
    if (!c || !o) return HG_EINVAL;
    const int64_t n = c->n;
    struct F {
        double *dst;
        const double *src;
        int64_t len;
    } f[] = {{o->mass, c->st.mass, n}, {o->pos, c->st.x, 3 * n},  {o->vel, c->st.v, 3 * n},
             {o->acc, c->st.a, 3 * n}, {o->jerk, c->st.j, 3 * n}, {o->snap, c->st.s, 3 * n},
             {o->crackle, c->st.c, 3 * n}, {o->t, c->st.t, n},    {o->dt, c->st.dt, n}};
    for (auto &q : f)
        if (q.dst) HG_CUDA(c, cudaMemcpyAsync(q.dst, q.src, q.len * sizeof(double), cudaMemcpyDefault, c->stream));
    int rc = sync_scalars(c);
    if (rc) return rc;
    o->t_sys = c->h_sc->t_cur;
    return HG_OK;
}

int hg_set_state(hg_ctx *c, const hg_state *in)
{
    const CallRange range_("hg_set_state");
    if (!c || !in) return HG_EINVAL;
    if (!in->mass || !in->pos || !in->vel || !in->acc || !in->jerk || !in->snap || !in->crackle || !in->t || !in->dt)
        return fail(c, HG_EINVAL, "every state field is required");
    if (!isfinite(in->t_sys)) return fail(c, HG_EINVAL, "t_sys must be finite");
    const int64_t n = c->n;
    struct F {
        double *dst;
        const double *src;
        int64_t len;
    } f[] = {{c->st2.mass, in->mass, n}, {c->st2.x, in->pos, 3 * n},  {c->st2.v, in->vel, 3 * n},
             {c->st2.a, in->acc, 3 * n}, {c->st2.j, in->jerk, 3 * n}, {c->st2.s, in->snap, 3 * n},
             {c->st2.c, in->crackle, 3 * n}, {c->st2.t, in->t, n},    {c->st2.dt, in->dt, n}};
    for (auto &q : f) HG_CUDA(c, cudaMemcpyAsync(q.dst, q.src, q.len * sizeof(double), cudaMemcpyDefault, c->stream));
    int32_t flag = 0;
    int rc = device_check(
        c,
        [&](int32_t *fl) {
            return launch_validate_state(c->st2, n, c->opts.dt_min, c->opts.dt_max, value_limits(c->mixed, c->eps), fl,
                                         c->stream);
        },
        &flag);
    if (rc) return rc;
    if (flag)
        return fail(c, HG_EINVAL,
                    "state check failed: masses > 0 and <= L min(1, eps^3), finite values within the limits "
                    "(mixed: L = 1e37, |positions| <= 1e15, other fields <= 1e30; FP64: L = 1e300, 1e150), dt a "
                    "power of two in [dt_min, dt_max], t a multiple of dt");
    // Copy into the live arrays (captured graphs keep their pointers).
    const State &d = c->st, &s = c->st2;
    struct G {
        double *dst;
        const double *src;
        int64_t len;
    } g[] = {{d.mass, s.mass, n}, {d.x, s.x, 3 * n}, {d.v, s.v, 3 * n}, {d.a, s.a, 3 * n}, {d.j, s.j, 3 * n},
             {d.s, s.s, 3 * n},   {d.c, s.c, 3 * n}, {d.t, s.t, n},     {d.dt, s.dt, n}};
    for (auto &q : g)
        HG_CUDA(c, cudaMemcpyAsync(q.dst, q.src, q.len * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    HG_CUDA(c, launch_tend(c->st, n, c->stream));
    c->tnext_valid = false;
    rc = upload_scalar(c, &c->d_sc->t_cur, in->t_sys);
    if (rc) return rc;
    invalidate(c);
    return HG_OK;
}

int hg_bind_device(hg_ctx *c, const hg_state *dev, int copy_in)
{
    const CallRange range_("hg_bind_device");
    if (!c) return HG_EINVAL;
    const int64_t n = c->n;
    auto copy_state = [&](const State &dst, const State &src) -> int {
        struct F {
            double *d;
            const double *s;
            int64_t len;
        } f[] = {{dst.mass, src.mass, n}, {dst.x, src.x, 3 * n}, {dst.v, src.v, 3 * n}, {dst.a, src.a, 3 * n},
                 {dst.j, src.j, 3 * n},   {dst.s, src.s, 3 * n}, {dst.c, src.c, 3 * n}, {dst.t, src.t, n},
                 {dst.dt, src.dt, n}};
        for (auto &q : f)
            if (q.d != q.s)
                HG_CUDA(c, cudaMemcpyAsync(q.d, q.s, q.len * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        return HG_OK;
    };
    int rc = HG_OK;
    if (!dev) {   // unbind: the state goes back into the context's own arrays
        if (!c->bound) return HG_OK;
        if ((rc = copy_state(c->own, c->st)) != HG_OK) return rc;
        c->st = c->own;
        c->bound = false;
    } else {
        double *p[9] = {dev->mass, dev->pos, dev->vel, dev->acc, dev->jerk, dev->snap, dev->crackle, dev->t, dev->dt};
        for (double *q : p) {
            cudaPointerAttributes a;
            if (!q || ((uintptr_t)q & 7u) != 0) return fail(c, HG_EINVAL, "every field must be an 8-byte aligned pointer");
            if (cudaPointerGetAttributes(&a, q) != cudaSuccess ||
                (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != c->device) {
                cudaGetLastError();
                return fail(c, HG_EINVAL, "every field must be device memory of the context's GPU");
            }
        }
        State b = c->st;
        b.mass = p[0]; b.x = p[1]; b.v = p[2]; b.a = p[3]; b.j = p[4]; b.s = p[5]; b.c = p[6]; b.t = p[7]; b.dt = p[8];
        b.tend = c->own.tend;
        if (copy_in) {
            if ((rc = copy_state(b, c->st)) != HG_OK) return rc;
        } else {
            int32_t flag = 0;
            rc = device_check(
                c,
                [&](int32_t *fl) {
                    return launch_validate_state(b, n, c->opts.dt_min, c->opts.dt_max, value_limits(c->mixed, c->eps), fl,
                                                 c->stream);
                },
                &flag);
            if (rc) return rc;
            if (flag) return fail(c, HG_EINVAL, "the bound arrays do not hold a valid state");
        }
        c->st = b;
        c->bound = true;
    }
    HG_CUDA(c, launch_tend(c->st, n, c->stream));
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->tnext_valid = false;
    drop_graphs(c);   // they captured the old state pointers
    invalidate(c);
    return HG_OK;
}

int hg_get_stats(hg_ctx *c, hg_stats *o)
{
    if (!c || !o) return HG_EINVAL;
    int rc = sync_scalars(c);
    if (rc) return rc;
    o->block_steps = c->h_sc->steps;
    o->interactions = c->h_sc->interactions;
    o->last_m = c->h_sc->m;
    o->t_sys = c->h_sc->t_cur;
    o->kernels = c->kernels;
    return HG_OK;
}

int hg_get_profile(hg_ctx *c, hg_profile *o, int reset)
{
    if (!c || !o) return HG_EINVAL;
    for (int q = 0; q < 5; ++q) o->ms[q] = c->prof_ms[q];
    o->block_steps = c->prof_steps;
    if (reset) {
        for (int q = 0; q < 5; ++q) c->prof_ms[q] = 0.0;
        c->prof_steps = 0;
    }
    return HG_OK;
}

int hg_tune(hg_ctx *c, int64_t m_max, int32_t reps, hg_tune_entry *report, int32_t cap, int32_t *n_out)
{
    const CallRange range_("hg_tune");
    if (!c) return HG_EINVAL;
    if (reps < 0 || reps > 1000) return fail(c, HG_EINVAL, "reps must be in [0, 1000]");
    if (cap < 0 || (cap > 0 && !report)) return fail(c, HG_EINVAL, "report capacity without a report array");
    if (n_out) *n_out = 0;
    PlanParams keep = c->pp;
    int rc = tune_impl(c, m_max, reps, report, cap, n_out);
    if (rc) {
        c->pp = keep;   // a failed run leaves the table as it was
        drop_graphs(c);
    }
    return rc;
}

int hg_time_evaluate(hg_ctx *c, const int32_t *idx, int64_t m, int32_t reps, double *us)
{
    const CallRange range_("hg_time_evaluate");
    if (!c || !us) return HG_EINVAL;
    if (isnan(c->t_pred)) return fail(c, HG_ESTATE, "hg_time_evaluate needs a preceding hg_predict");
    if (m < 1 || m > c->n || !idx) return fail(c, HG_EINVAL, "m must be in [1, n] and idx given");
    if (reps < 0 || reps > 1000) return fail(c, HG_EINVAL, "reps must be in [0, 1000]");
    if (is_device_ptr(idx)) {
        HG_CUDA(c, cudaMemcpyAsync(c->d_idx2, idx, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
        int32_t flag = 0;
        int rc = device_check(c, [&](int32_t *f) { return launch_validate_idx(c->d_idx2, m, c->n, f, c->stream); },
                              &flag);
        if (rc) return rc;
        if (flag) return fail(c, HG_EINVAL, "idx must be strictly increasing and in [0, n)");
    } else {
        for (int64_t q = 0; q < m; ++q)
            if (idx[q] < 0 || idx[q] >= c->n || (q > 0 && idx[q] <= idx[q - 1]))
                return fail(c, HG_EINVAL, "idx must be strictly increasing and in [0, n)");
        HG_CUDA(c, cudaMemcpyAsync(c->d_idx2, idx, m * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    }
    int32_t *t = c->d_idx;
    c->d_idx = c->d_idx2;
    c->d_idx2 = t;
    drop_graphs(c);   // they captured the old list pointer
    const double t_pred = c->t_pred;
    invalidate(c);    // the results buffers are overwritten: no evaluation is pending
    c->t_pred = t_pred;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HG_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, HG_ECUDA, "cudaEventCreate failed");
    }
    int r = reps;
    int rc = time_eval(c, m, &r, e0, e1, us);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return sync_scalars(c);
}

int hg_get_tuning(hg_ctx *c, int16_t *table)
{
    if (!c || !table) return HG_EINVAL;
    for (int k = 0; k < kTuneBuckets; ++k) table[k] = c->pp.tuned[k];
    return HG_OK;
}

int hg_set_tuning(hg_ctx *c, const int16_t *table)
{
    if (!c || !table) return HG_EINVAL;
    for (int k = 0; k < kTuneBuckets; ++k) {
        const int v = table[k];
        const bool ok = v == -1 || (c->bv.nc > 0 ? batch_code_ok(v) : (v >= 0 && v < plan_total(c->pp)));
        if (!ok) return fail(c, HG_EINVAL, "tuning table value out of range for this context");
    }
    for (int k = 0; k < kTuneBuckets; ++k) c->pp.tuned[k] = table[k];
    drop_graphs(c);
    return HG_OK;
}

int hg_test_corrupt_list(hg_ctx *c, int64_t pos, int32_t value)
{
    if (!c) return HG_EINVAL;
#if defined(HG_CHECKED)
    const CallRange range_("hg_test_corrupt_list");
    if (c->cur_m < 1 || pos < 0 || pos >= c->cur_m) return fail(c, HG_EINVAL, "pos must lie in the current block");
    HG_CUDA(c, cudaMemcpyAsync(c->d_idx + pos, &value, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    HG_CUDA(c, cudaStreamSynchronize(c->stream));
    return HG_OK;
#else
    (void)pos;
    (void)value;
    return fail(c, HG_EINVAL, "hg_test_corrupt_list exists only in the checked build (HG_CHECKED)");
#endif
}

int hg_build_checked(void)
{
#if defined(HG_CHECKED)
    return 1;
#else
    return 0;
#endif
}

int hg_inject_fault(int32_t kind, int64_t nth)
{
    if (kind != HG_FAULT_NONE && kind != HG_FAULT_ALLOC && kind != HG_FAULT_CUDA) return HG_EINVAL;
    if (kind != HG_FAULT_NONE && nth < 1) return HG_EINVAL;
    g_fault_kind.store(HG_FAULT_NONE);
    g_fault_left.store(kind == HG_FAULT_NONE ? 0 : nth);
    g_fault_kind.store(kind);
    return HG_OK;
}

int64_t hg_size(const hg_ctx *c) { return c ? c->n : 0; }

const char *hg_last_error(const hg_ctx *c) { return c ? c->err.c_str() : ""; }

void hg_free(hg_ctx *c) { release(c); }

}  // extern "C"
