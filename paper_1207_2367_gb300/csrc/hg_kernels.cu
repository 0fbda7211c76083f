// hg_kernels.cu -- the FP64 parts of a block step (next-block selection,
// predictor, corrector with the time-step update), start-up, energy and
// input validation.  Sect. 3 of the HiGPUs paper; Table 1 sections 1, 2, 8.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hg_kernels.cuh"

namespace hg {
namespace {

constexpr int kNBThreads = 256;

__device__ __forceinline__ int64_t block_sum_i64(int64_t v, int64_t *sh)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (l == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

// ------------------------------------------------------------------------
// Table 1 section 1: next block time and the ascending list of due particles.
// Times are dyadic and non-negative, so tend_i = t_i + dt_i is exact and its
// IEEE bit pattern orders like its value: the passes compare 64-bit integers.
// One CTA per contiguous chunk; the last CTA to finish a pass (atomic arrival
// count, no waiting) completes it: pass 1 the global minimum, pass 2 the
// chunk offsets, m and the evaluation plan.  Results do not depend on the
// order in which CTAs run.
// ------------------------------------------------------------------------
__device__ __forceinline__ long long block_min_ll(long long v, long long *sh)
{
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : LLONG_MAX;
        for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (l == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

// The evaluation plan for block size m, by every thread of one CTA (at least
// kPlanCandidates threads would score one candidate each; fewer loop): the
// lowest cost wins, ties to the lowest candidate index (make_plan's choice on
// the host).  A tuned candidate of m's bucket that is admissible wins outright.
__device__ void plan_on_block(int64_t m, const PlanParams &q, DevScalars *sc)
{
    __shared__ int64_t s_cost[32];
    __shared__ int s_cand[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    Plan p;
    const int tc = q.tuned[tune_bucket(m)];
    if (tc >= 0 && plan_candidate(m, q, tc, p) >= 0) {   // measured choice
        if (threadIdx.x == 0) *reinterpret_cast<Plan *>(sc->plan) = p;
        return;
    }
    int64_t best = -1;
    int bc = 0x7fffffff;
    for (int c = threadIdx.x; c < plan_total(q); c += blockDim.x) {
        const int64_t cost = plan_candidate(m, q, c, p);
        if (cost >= 0 && (best < 0 || cost < best)) {
            best = cost;
            bc = c;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const int64_t ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
        if (ob >= 0 && (best < 0 || ob < best || (ob == best && oc < bc))) {
            best = ob;
            bc = oc;
        }
    }
    if (lane == 0) {
        s_cost[w] = best;
        s_cand[w] = bc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k) {
            const int64_t ob = s_cost[k];
            const int oc = s_cand[k];
            if (ob >= 0 && (best < 0 || ob < best || (ob == best && oc < bc))) {
                best = ob;
                bc = oc;
            }
        }
        plan_candidate(m, q, best >= 0 ? bc : 0, p);
        *reinterpret_cast<Plan *>(sc->plan) = p;
    }
}


// True in every thread of the CTA that arrives last (counter reset for reuse).
__device__ __forceinline__ bool last_to_arrive(uint32_t *counter, uint32_t total, int *sh_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(counter, 1u);
        *sh_flag = (prev == total - 1) ? 1 : 0;
        if (*sh_flag) {
            *counter = 0u;
            __threadfence();
        }
    }
    __syncthreads();
    return *sh_flag != 0;
}

__global__ void __launch_bounds__(kNBThreads) k_nb_min(const double *tend, int64_t n, int64_t chunk,
                                                       long long *part, int g, DevScalars *sc)
{
    __shared__ long long sh[32];
    __shared__ int last;
    const long long *bits = reinterpret_cast<const long long *>(tend);
    const int64_t lo = blockIdx.x * chunk, hi = (lo + chunk < n) ? lo + chunk : n;
    long long v = LLONG_MAX;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v = min(v, __ldg(bits + i));
    v = block_min_ll(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
    if (!last_to_arrive(&sc->arrive[0], (uint32_t)g, &last)) return;
    __threadfence();
    v = LLONG_MAX;
    for (int c = threadIdx.x; c < g; c += blockDim.x) v = min(v, *((volatile long long *)part + c));
    v = block_min_ll(v, sh);
    if (threadIdx.x == 0) sc->tnext_bits = v;
}

__global__ void __launch_bounds__(kNBThreads) k_nb_count(const double *tend, int64_t n, int64_t chunk,
                                                         int32_t *cnt, int32_t *off, int g, DevScalars *sc,
                                                         int count_step, const PlanParams pq)
{
    __shared__ long long shl[32];
    __shared__ int64_t shi[32];
    __shared__ int last;
    const long long tn = *((volatile long long *)&sc->tnext_bits);
    const long long *bits = reinterpret_cast<const long long *>(tend);
    const int64_t lo = blockIdx.x * chunk, hi = (lo + chunk < n) ? lo + chunk : n;
    int64_t c = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c += (__ldg(bits + i) == tn) ? 1 : 0;
    c = block_sum_i64(c, shi);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (int32_t)c;
    if (!last_to_arrive(&sc->arrive[1], (uint32_t)g, &last)) return;
    __threadfence();
    // Exclusive prefix of the chunk counts: each thread scans a run of chunks.
    const int per = (g + (int)blockDim.x - 1) / (int)blockDim.x;
    const int c0 = threadIdx.x * per, c1 = (c0 + per < g) ? c0 + per : g;
    int64_t run = 0;
    for (int k = c0; k < c1; ++k) run += *((volatile int32_t *)cnt + k);
    // block exclusive scan of the runs
    int64_t incl = run;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += u;
    }
    __syncthreads();
    if (l == 31) shi[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t x = (l < (int)(blockDim.x >> 5)) ? shi[l] : 0;
        int64_t xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, xi, o);
            if (l >= o) xi += u;
        }
        shi[l] = xi - x;   // exclusive warp offsets
        if (l == 31) shl[0] = xi;   // total
    }
    __syncthreads();
    int64_t base = shi[w] + incl - run;
    for (int k = c0; k < c1; ++k) {
        off[k] = (int32_t)base;
        base += *((volatile int32_t *)cnt + k);
    }
    const int64_t tot = shl[0];
    const double t_next = __longlong_as_double(tn);
    const bool take = t_next <= sc->t_stop;
    if (threadIdx.x == 0) {
        if (take) {
            sc->m = tot;
            sc->t_cur = t_next;
            sc->done = 0;
            if (count_step) {   // 1: count the step and m n interactions; 2: the step only
                sc->steps += 1;
                if (count_step == 1) sc->interactions += tot * n;
            }
        } else {
            sc->m = 0;
            sc->done = 1;
        }
    }
    if (take) plan_on_block(tot, pq, sc);   // uniform branch: every thread of the CTA
}

__global__ void __launch_bounds__(kNBThreads) k_nb_scatter(const double *tend, int64_t n, int64_t chunk,
                                                           const int32_t *off, int32_t *idx, const DevScalars *sc)
{
    __shared__ int32_t woff[33];
    if (*((volatile int64_t *)&sc->m) <= 0) return;
    const long long tn = *((volatile long long *)&sc->tnext_bits);
    const long long *bits = reinterpret_cast<const long long *>(tend);
    int64_t pre = off[blockIdx.x];
    const int64_t lo = blockIdx.x * chunk, hi = (lo + chunk < n) ? lo + chunk : n;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool due = (i < hi) && (__ldg(bits + i) == tn);
        const unsigned ball = __ballot_sync(0xffffffffu, due);
        if (l == 0) woff[w] = __popc(ball);
        __syncthreads();
        if (w == 0) {
            const int v = (l < (int)(blockDim.x >> 5)) ? woff[l] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (l >= o) incl += u;
            }
            woff[l] = incl - v;
            if (l == 31) woff[32] = incl;
        }
        __syncthreads();
        if (due) idx[pre + woff[w] + __popc(ball & ((1u << l) - 1u))] = (int32_t)i;
        pre += woff[32];
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// Sect. 3 item 1: Taylor predictor through crackle, FP64, h = t - t_j.
// ------------------------------------------------------------------------
struct Pred {
    double x[3], v[3], a[3];
};

__device__ __forceinline__ Pred predict_one(const State &st, int64_t i, double tt)
{
    Pred p;
    const double h = tt - st.t[i];
    const double h2 = h * h * 0.5;              // h^2/2
    const double h3 = h2 * h * (1.0 / 3.0);     // h^3/6
    const double h4 = h3 * h * 0.25;            // h^4/24
    const double h5 = h4 * h * 0.2;             // h^5/120
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t q = 3 * i + k;
        const double x = st.x[q], v = st.v[q], a = st.a[q], j = st.j[q], s = st.s[q], c = st.c[q];
        p.x[k] = x + fma(h, v, fma(h2, a, fma(h3, j, fma(h4, s, h5 * c))));
        p.v[k] = v + fma(h, a, fma(h2, j, fma(h3, s, h4 * c)));
        p.a[k] = a + fma(h, j, fma(h2, s, h3 * c));
    }
    return p;
}

// Record r from particle i predicted to time tt (i >= n: a padding record).
template <bool MIXED>
__device__ __forceinline__ void predict_record(const State &st, const Records &rec, int64_t i, int64_t n, int64_t r,
                                               double tt)
{
    {
        if (MIXED) {
            MixedRecord v;
            if (i < n) {
                // Positions: x + h v in FP64 plus the rest of the Taylor series,
                // h^2 (a/2 + h (j/6 + h (s/24 + h c/120))), as an FP32 Horner
                // series (its rounding, ~5e-7 of a term that is itself a small
                // part of the step's displacement, stays far below the FP32 pair
                // error), then split into float hi + lo: 3 FP64 instructions per
                // component, the FP64 pipe being this kernel's limit on GB300.
                // Velocities and accelerations feed only the FP32 pair
                // arithmetic: FP32 Horner series from the rounded derivatives.
                const double h = tt - st.t[i];
                const float hf = d2f(h);
                float hi[3], lo[3], vp[3], ap[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int64_t q = 3 * i + k;
                    const double x = st.x[q], v = st.v[q], a = st.a[q], j = st.j[q], s = st.s[q], c = st.c[q];
                    const float vf = d2f(v), af = d2f(a), jf = d2f(j), sf = d2f(s), cf = d2f(c);
                    const float rest =
                        hf * hf *
                        fmaf(hf, fmaf(hf, fmaf(hf, cf * (1.f / 120.f), sf * (1.f / 24.f)), jf * (1.f / 6.f)), af * 0.5f);
                    const double xp = fma(h, v, x) + f2d(rest);
                    hi[k] = d2f(xp);
                    lo[k] = d2f(xp - f2d(hi[k]));
                    vp[k] = fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, cf * (1.f / 24.f), sf * (1.f / 6.f)), jf * 0.5f), af),
                                 vf);
                    ap[k] = fmaf(hf, fmaf(hf, fmaf(hf, cf * (1.f / 6.f), sf * 0.5f), jf), af);
                }
                v = MixedRecord{hi[0], hi[1], hi[2], d2f(st.mass[i]), lo[0], lo[1], lo[2], ap[0],
                                vp[0], vp[1], vp[2], ap[1], ap[2]};
            } else {
                const float far = (float)kPadCoord;
                v = MixedRecord{far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            }
            store_mixed_record(rec, r, v);
        } else {
            double2 q0, q1, q2, q3, q4;
            if (i < n) {
                const Pred p = predict_one(st, i, tt);
                q0 = make_double2(p.x[0], p.x[1]);
                q1 = make_double2(p.x[2], st.mass[i]);
                q2 = make_double2(p.v[0], p.v[1]);
                q3 = make_double2(p.v[2], p.a[0]);
                q4 = make_double2(p.a[1], p.a[2]);
            } else {
                q0 = make_double2(kPadCoord, kPadCoord);
                q1 = make_double2(kPadCoord, 0.0);
                q2 = q3 = q4 = make_double2(0.0, 0.0);
            }
            static_cast<double2 *>(rec.p[0])[r] = q0;
            static_cast<double2 *>(rec.p[1])[r] = q1;
            static_cast<double2 *>(rec.p[2])[r] = q2;
            static_cast<double2 *>(rec.p[3])[r] = q3;
            static_cast<double2 *>(rec.p[4])[r] = q4;
        }
    }
}

// Single system: record i is particle i (padding beyond n).  Clusters:
// particle i goes to record rmap[i]; padding slots were written at set-up.
template <bool MIXED>
__global__ void k_predict(const State st, const Records rec, int64_t n, int64_t npad, const double *t_dev,
                          double t_host, const int64_t *m_dev, const int32_t *rmap)
{
    if (m_dev && *m_dev <= 0) return;
    const double tt = t_dev ? *t_dev : t_host;
    const int64_t count = rmap ? n : npad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        predict_record<MIXED>(st, rec, i, n, rmap ? (int64_t)rmap[i] : i, tt);
}

// Clusters, in a block step: only the clusters with active particles need
// predicted data.  Work index w in [0, pred_off[nc]) is particle
// cl_off[c] + (w - pred_off[c]) of the cluster c whose range holds w.
template <bool MIXED>
__global__ void k_predict_clusters(const State st, const Records rec, int64_t n, BatchView bv, const double *t_dev,
                                   const int64_t *m_dev)
{
    if (*m_dev <= 0) return;
    const double tt = *t_dev;
    const int64_t total = bv.pred_off[bv.nc];
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = bv.nc - 1;   // last cluster with pred_off[c] <= w
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bv.pred_off[mid] <= w) lo = mid; else hi = mid - 1;
        }
        const int64_t i = bv.cl_off[lo] + (w - bv.pred_off[lo]);
        predict_record<MIXED>(st, rec, i, n, bv.rmap[i], tt);
    }
}

// One system, graph-replayed block steps: Table 1 sections 1 and 2 in one
// pass.  sc->tnext_bits holds min_i tend_i of the current state (left by the
// previous correction).  Every thread predicts its records to t_next and the
// due particles (tend_i == t_next, exact integer compare) are appended to idx
// with one atomic per warp: the list order is arbitrary, which changes nothing
// computed (a particle's sums do not depend on its position in the list).  The
// last CTA to finish (arrival count, no waiting) publishes m, the block time,
// the counters and the evaluation plan, and clears the minimum for the next
// correction.  t_next > t_stop: no step (m = 0, done).
template <bool MIXED>
__global__ void __launch_bounds__(256) k_predict_select(const State st, const Records rec, int64_t n, int64_t npad,
                                                       int32_t *idx, DevScalars *sc, int count_step,
                                                       const PlanParams pq)
{
    __shared__ int last;
    const long long tn = *((volatile long long *)&sc->tnext_bits);
    const double t_next = __longlong_as_double(tn);
    if (!(t_next <= *((volatile double *)&sc->t_stop))) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sc->m = 0;
            sc->done = 1;
        }
        return;
    }
    const long long *bits = reinterpret_cast<const long long *>(st.tend);
    const int l = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < npad; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        if (i < npad) predict_record<MIXED>(st, rec, i, n, i, t_next);
        const bool due = i < n && bits[i] == tn;
        const unsigned ball = __ballot_sync(0xffffffffu, due);
        if (ball) {
            uint32_t b0 = 0;
            if (l == 0) b0 = atomicAdd(&sc->slot, (uint32_t)__popc(ball));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            const int64_t at = (int64_t)b0 + __popc(ball & ((1u << l) - 1u));
            if (due) {
                if (at < n) idx[at] = (int32_t)i;
                else atomicOr(&sc->err, ERR_STATE);   // unreachable while slot starts at 0
            }
        }
    }
    if (!last_to_arrive(&sc->arrive[2], gridDim.x, &last)) return;
    __threadfence();
    // One read of the slot count, shared before thread 0 resets it (a thread
    // reading it after the reset would score the plan for another m).
    __shared__ int64_t s_m;
    if (threadIdx.x == 0) s_m = (int64_t)*((volatile uint32_t *)&sc->slot);
    __syncthreads();
    const int64_t m = s_m;
    if (threadIdx.x == 0) {
        sc->m = m;
        sc->t_cur = t_next;
        sc->done = 0;
        sc->steps += 1;
        if (count_step == 1) sc->interactions += m * n;
        sc->slot = 0u;
        sc->tnext_bits = LLONG_MAX;
    }
    plan_on_block(m > 0 ? m : 1, pq, sc);
}

// Predicted FP64 positions and velocities (energy diagnostics).
__global__ void k_predict_xv(const State st, int64_t n, double tt, double *xe, double *ve)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Pred p = predict_one(st, i, tt);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            xe[3 * i + k] = p.x[k];
            ve[3 * i + k] = p.v[k];
        }
    }
}

// ------------------------------------------------------------------------
// Time steps: generalized Aarseth criterion and power-of-two blocks.
// ------------------------------------------------------------------------
__device__ __forceinline__ double norm3(const double *p)
{
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(p[0], p[0]), __dmul_rn(p[1], p[1])), __dmul_rn(p[2], p[2])));
}

// eta (A^(1)/A^(p-2))^(1/(p-3)) with A^(s) = sqrt(|a^(s-1)||a^(s+1)| + |a^(s)|^2);
// d holds a^(0..p-1) (p = 4 or 6).
__device__ double criterion(double eta, int p, const double (*d)[3])
{
    double nr[6];
    for (int s = 0; s < p; ++s) nr[s] = norm3(d[s]);
    const double A1 = sqrt(__dadd_rn(__dmul_rn(nr[0], nr[2]), __dmul_rn(nr[1], nr[1])));
    const double Ap = sqrt(__dadd_rn(__dmul_rn(nr[p - 3], nr[p - 1]), __dmul_rn(nr[p - 2], nr[p - 2])));
    if (Ap == 0.0) return INFINITY;
    const double ratio = A1 / Ap;
    return (p == 4) ? eta * ratio : eta * cbrt(ratio);
}

// Shrink to the largest 2^k <= crit; grow x2 only when t_new is a multiple of
// the doubled step; clamp to [dt_min, dt_max].
__device__ double block_dt(double crit, double dt, double t_new, double dt_min, double dt_max)
{
    if (crit < dt) {
        while (dt > crit && dt > dt_min) dt *= 0.5;
    } else if (crit >= 2.0 * dt && 2.0 * dt <= dt_max && fmod(t_new, 2.0 * dt) == 0.0) {
        dt *= 2.0;
    }
    return fmin(fmax(dt, dt_min), dt_max);
}

__device__ double block_dt_init(double crit, double dt_min, double dt_max)
{
    double dt = dt_max;
    while (dt > crit && dt > dt_min) dt *= 0.5;
    return dt;
}

// Start-up: store a, jerk, snap of the full evaluation, crackle = 0, t = 0 and
// the first step from the p = 4 criterion with eta_init.
__global__ void k_start(State st, int64_t n, const double *ra, const double *rj, const double *rs, StepParams sp)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d[4][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d[0][k] = ra[3 * i + k];
            d[1][k] = rj[3 * i + k];
            d[2][k] = rs[3 * i + k];
            d[3][k] = 0.0;
            st.a[3 * i + k] = d[0][k];
            st.j[3 * i + k] = d[1][k];
            st.s[3 * i + k] = sp.order == 4 ? 0.0 : d[2][k];   // the 4th-order scheme keeps a, jerk
            st.c[3 * i + k] = 0.0;
        }
        st.t[i] = 0.0;
        st.dt[i] = block_dt_init(criterion(sp.eta_init, 4, d), sp.dt_min, sp.dt_max);
        st.tend[i] = st.dt[i];
    }
}

// ------------------------------------------------------------------------
// Sect. 3 item 3: corrector, Hermite interpolation for crackle/pop/a^(5),
// p = 6 criterion and the new block step, for the m particles of the block.
// ------------------------------------------------------------------------

// Exact powers of two from integer exponents (no FP64 instruction on the
// normal range; GB300 issues a warp-wide FP64 instruction in ~64 cycles, so the
// corrector's latency is its count of dependent FP64 instructions).
__device__ __forceinline__ double pow2i(int e)
{
    if (e > 1023) return INFINITY;
    if (e < -1022) return ldexp(1.0, e);
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Exponent k of h = 2^k (normal, positive); false if h is not such a power of two.
__device__ __forceinline__ bool pow2_exponent(double h, int &k)
{
    const long long b = __double_as_longlong(h);
    const int be = (int)((b >> 52) & 0x7ff);
    if (b <= 0 || be == 0 || be == 0x7ff || (b & 0xfffffffffffffLL) != 0) return false;
    k = be - 1023;
    return true;
}

// Component k of particle i over its step h: corrected v and r (stored, with
// the new a, jerk, snap and crackle), and crackle, pop and a^(5) from the
// degree-5 interpolant through a, jerk, snap at both ends of the step.
// h = 2^e: h/2, h^2/10 = 2^(2e) fl(1/10), h^3/120 = 2^(3e) fl(1/120) and the
// reciprocal powers are exact scalings, equal to the divisions they replace.
__device__ __forceinline__ void correct_component(const State &st, int64_t i, int k, double h, int e, bool pow2,
                                                  double a1, double j1, double s1, double &c3, double &c4, double &c5,
                                                  double &Ak)
{
    double hh, h2, h3, ih3, ih4, ih5;
    if (pow2) {
        hh = pow2i(e - 1);
        h2 = pow2i(2 * e) * 0.1;
        h3 = pow2i(3 * e) * (1.0 / 120.0);
        ih3 = pow2i(-3 * e);
        ih4 = pow2i(-4 * e);
        ih5 = pow2i(-5 * e);
    } else {
        hh = h / 2.0;
        h2 = h * h / 10.0;
        h3 = h * h * h / 120.0;
        const double ih = 1.0 / h;
        ih3 = ih * ih * ih;
        ih4 = ih3 * ih;
        ih5 = ih4 * ih;
    }
    const int64_t q = 3 * i + k;
    const double x0 = st.x[q], v0 = st.v[q], a0 = st.a[q], j0 = st.j[q], s0 = st.s[q];
    const double v1 = v0 + hh * (a1 + a0) - h2 * (j1 - j0) + h3 * (s1 + s0);
    const double x1 = x0 + hh * (v1 + v0) - h2 * (a1 - a0) + h3 * (j1 + j0);
    const double A = a1 - a0 - j0 * h - s0 * h * h / 2.0;
    const double J = (j1 - j0 - s0 * h) * h;
    const double S = (s1 - s0) * h * h;
    c3 = (60.0 * A - 36.0 * J + 9.0 * S) * ih3;
    c4 = (360.0 * A - 192.0 * J + 36.0 * S) * ih4;
    c5 = (720.0 * A - 360.0 * J + 60.0 * S) * ih5;
    Ak = A;
    st.x[q] = x1;
    st.v[q] = v1;
    st.a[q] = a1;
    st.j[q] = j1;
    st.s[q] = s1;
    st.c[q] = c3;
}

// 4th-order scheme, component k of particle i (the two-point Hermite corrector
// and the cubic interpolant through a and jerk at both ends): corrected v and r,
// new a and jerk (snap and crackle stored as zero: the predictor ends at jerk),
// and snap and crackle at the step's end for the p = 4 criterion.  h = 2^e:
// h^2/12 = 2^(2e) fl(1/12) and the reciprocal powers are exact scalings.
__device__ __forceinline__ void correct4_component(const State &st, int64_t i, int k, double h, int e, bool pow2,
                                                   double a1, double j1, double &s1, double &c1, double &Ak)
{
    double hh, h2, ih2, ih3;
    if (pow2) {
        hh = pow2i(e - 1);
        h2 = pow2i(2 * e) * (1.0 / 12.0);
        ih2 = pow2i(-2 * e);
        ih3 = pow2i(-3 * e);
    } else {
        hh = h / 2.0;
        h2 = h * h / 12.0;
        ih2 = 1.0 / (h * h);
        ih3 = ih2 / h;
    }
    const int64_t q = 3 * i + k;
    const double x0 = st.x[q], v0 = st.v[q], a0 = st.a[q], j0 = st.j[q];
    const double v1 = v0 + hh * (a0 + a1) + h2 * (j0 - j1);
    const double x1 = x0 + hh * (v0 + v1) + h2 * (a0 - a1);
    const double c = (12.0 * (a0 - a1) + 6.0 * h * (j0 + j1)) * ih3;
    const double s0 = (-6.0 * (a0 - a1) - h * (4.0 * j0 + 2.0 * j1)) * ih2;
    s1 = s0 + c * h;
    c1 = c;
    Ak = a1 - a0 - j0 * h;
    st.x[q] = x1;
    st.v[q] = v1;
    st.a[q] = a1;
    st.j[q] = j1;
    st.s[q] = 0.0;
    st.c[q] = 0.0;
}

// ---- FP32 estimate of floor(log2 crit) for the step criterion --------------
// Logarithms are carried as e + r: an exact integer e and a small float r, so
// that exponents up to +-2046 keep ~1e-7 absolute precision.  Every step below
// (mantissa truncated to 24 bits, lg2/ex2 approximations) errs by < 1e-6 in
// log2 units; an estimate within kLogGuard of an integer is decided by the FP64
// criterion instead, so the step chosen is always the FP64 criterion's.
struct Log2 {
    int e;
    float r;
};
constexpr float kLogGuard = 1.0e-4f;

__device__ __forceinline__ bool log2_of(double q, Log2 &o)
{
    const long long b = __double_as_longlong(q);
    const int be = (int)((b >> 52) & 0x7ff);
    if (b <= 0 || be == 0 || be == 0x7ff) return false;   // zero, negative, subnormal, inf, nan
    o.e = be - 1023;
    o.r = __log2f(__int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff)));   // mantissa in [1, 2)
    return true;
}
__device__ __forceinline__ Log2 l2_add(Log2 a, Log2 b) { return Log2{a.e + b.e, a.r + b.r}; }
// x / d for d = 2, 3 or 6: e = d k + j (floor division), x / d = k + (j + r) / d.
__device__ __forceinline__ Log2 l2_div(Log2 a, int d)
{
    int k = a.e / d, j = a.e - k * d;
    if (j < 0) {
        j += d;
        k -= 1;
    }
    return Log2{k, ((float)j + a.r) / (float)d};
}
// log2(2^a + 2^b)
__device__ __forceinline__ Log2 l2_sum(Log2 a, Log2 b)
{
    float d = (float)(a.e - b.e) + (a.r - b.r);
    if (d < 0.0f) {
        const Log2 t = a;
        a = b;
        b = t;
        d = -d;
    }
    if (d > 60.0f) return a;
    return Log2{a.e, a.r + __log2f(1.0f + exp2f(-d))};
}

// floor(log2(eta (A1 / A_{p-2})^(1/(p-3)))) for p = 4 or 6, with A1 = sqrt(n0 n2 +
// n1^2), A_{p-2} = sqrt(n_{p-3} n_{p-1} + n_{p-2}^2), n_s = |d_s|, from the
// squared norms q_s; false when undecided (a q_s that is zero or not normal, or
// the estimate within kLogGuard of an integer).
template <int P>
__device__ __forceinline__ bool criterion_floor_log2(const double *qn, float log2_eta, int &F)
{
    Log2 l[P];
#pragma unroll
    for (int s = 0; s < P; ++s)
        if (!log2_of(qn[s], l[s])) return false;
    // log2 A^2 terms: log2(n0 n2) = (L0 + L2) / 2, log2(n1^2) = L1 (L = log2 q).
    const Log2 A1sq = l2_sum(l2_div(l2_add(l[0], l[2]), 2), l[1]);
    const Log2 Apsq = l2_sum(l2_div(l2_add(l[P - 3], l[P - 1]), 2), l[P - 2]);
    // log2 crit = log2 eta + (log2 A1^2 - log2 A_{p-2}^2) / (2 (p - 3))
    const Log2 x = l2_div(Log2{A1sq.e - Apsq.e, A1sq.r - Apsq.r}, 2 * (P - 3));
    const float y = log2_eta + x.r;
    const float fy = floorf(y);
    const float frac = y - fy;
    if (frac < kLogGuard || frac > 1.0f - kLogGuard) return false;
    F = x.e + (int)fy;
    return true;
}

// t1 (>= 0, dyadic) is an integer multiple of 2^p: the lowest set bit of its
// significand weighs at least 2^p.  Subnormal t1: fmod.
__device__ __forceinline__ bool multiple_of_pow2(double t1, int p)
{
    if (t1 == 0.0) return true;
    const long long b = __double_as_longlong(t1);
    const int be = (int)((b >> 52) & 0x7ff);
    if (be == 0 || b < 0) return fmod(t1, pow2i(p)) == 0.0;
    const long long mant = (b & 0xfffffffffffffLL) | (1LL << 52);
    return (be - 1023 - 52) + (__ffsll(mant) - 1) >= p;
}

__device__ __forceinline__ double sq3(const double *p) { return p[0] * p[0] + p[1] * p[1] + p[2] * p[2]; }

// New time and p = 6 step of particle i from d = a^(0..5) at the step's end.
// A: the acceleration change left after a0 + j0 h + s0 h^2/2 (a0 + j0 h for
// p = 4).  Below the noise floor of the evaluation, sp.noise_rel times the
// noise scale (sum_j m_j / r_ij^2 where the evaluation provides it, else |a1|;
// compared as squares), the interpolated derivatives are noise and the
// criterion may not shrink the step.
template <int P>
__device__ __forceinline__ double finish_step(const State &st, int64_t i, double h, int e, bool pow2,
                                              const double (*d)[3], const double *A, double scale2,
                                              const StepParams &sp, bool store)
{
    const double t1 = st.t[i] + h;
    const bool noisy = sp.noise_rel > 0.0 && sq3(A) < (sp.noise_rel * sp.noise_rel) * scale2;
    double dt1;
    int F, kmin, kmax;
    double qn[P];
#pragma unroll
    for (int s = 0; s < P; ++s) qn[s] = sq3(d[s]);
    if (pow2 && pow2_exponent(sp.dt_min, kmin) && pow2_exponent(sp.dt_max, kmax) &&
        (noisy || criterion_floor_log2<P>(qn, sp.log2_eta, F))) {
        // The power-of-two rule (block_dt) on exponents: shrink to max(F, k_min)
        // when crit < h, double when crit >= 2h, 2h <= dt_max and t1 is a
        // multiple of 2h; clamp to [dt_min, dt_max].
        int kn = e;
        if (!noisy && F < e) {
            kn = F > kmin ? F : kmin;
        } else if ((noisy || F >= e + 1) && e + 1 <= kmax && multiple_of_pow2(t1, e + 1)) {
            kn = e + 1;
        }
        kn = kn < kmin ? kmin : (kn > kmax ? kmax : kn);
        dt1 = pow2i(kn);
    } else {
        double crit = criterion(sp.eta, P, d);
        if (noisy) crit = INFINITY;
        dt1 = block_dt(crit, h, t1, sp.dt_min, sp.dt_max);
    }
    if (store) {
        st.t[i] = t1;
        st.dt[i] = dt1;
        st.tend[i] = t1 + dt1;
    }
    return t1 + dt1;
}

// Three lanes per particle, one per component: warp w takes units of 10
// particles (lanes 3p, 3p+1, 3p+2 hold particle p of the unit; lanes 30 and 31
// idle).  Each lane corrects its component; shuffles then give every lane of the
// triple all components, and the three run the same step logic on the same
// values (the first stores the new time and step).  The chain of dependent FP64
// instructions of a small block is a third of the one-thread-per-particle form.
constexpr int kCorrUnit = 10;

template <int P>
__device__ __forceinline__ void correct_lane(const State &st, const int32_t *idx, const double *ra, const double *rj,
                                             const double *rs, const double *rn, const StepParams &sp, int64_t m, int64_t n, int32_t *err,
                                             int64_t u, long long &low)
{
    const int lane = threadIdx.x & 31, sub = lane / 3, k = lane - 3 * sub;
    const int64_t q = u * kCorrUnit + sub;
    bool act = sub < kCorrUnit && q < m;
    if (act && !in_bounds(idx[q] >= 0 && (int64_t)idx[q] < n, err)) act = false;
    double dk[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, Ak = 0.0, h = 1.0;
    int64_t i = 0;
    int e = 0;
    bool pow2 = false;
    if (act) {
        i = idx[q];
        h = st.dt[i];
        pow2 = pow2_exponent(h, e);
        dk[0] = ra[3 * q + k];
        dk[1] = rj[3 * q + k];
        if (P == 4) {
            correct4_component(st, i, k, h, e, pow2, dk[0], dk[1], dk[2], dk[3], Ak);
        } else {
            dk[2] = rs[3 * q + k];
            correct_component(st, i, k, h, e, pow2, dk[0], dk[1], dk[2], dk[3], dk[4], dk[5], Ak);
        }
    }
    double d[6][3], A[3];
    const int base = 3 * sub;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int src = base + c < 32 ? base + c : 31;
#pragma unroll
        for (int r = 0; r < P; ++r) d[r][c] = __shfl_sync(0xffffffffu, dk[r], src);
        A[c] = __shfl_sync(0xffffffffu, Ak, src);
    }
    if (act) {
        const double scale2 = rn ? rn[q] * rn[q] : sq3(d[0]);
        low = min(low, __double_as_longlong(finish_step<P>(st, i, h, e, pow2, d, A, scale2, sp, k == 0)));
    }
}

__global__ void __launch_bounds__(128) k_correct(State st, const int32_t *idx, const int64_t *m_dev, int64_t m_host,
                                                 const double *ra, const double *rj, const double *rs,
                                                 const double *rn, StepParams sp, DevScalars *sc, int64_t n,
                                                 int min_pass)
{
    __shared__ long long sh[32];
    const int64_t m = m_dev ? *m_dev : m_host;
    if (m <= 0) return;
    long long low = LLONG_MAX;
    const int64_t units = (m + kCorrUnit - 1) / kCorrUnit;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += nw) {   // warp-uniform
        if (sp.order == 4)
            correct_lane<4>(st, idx, ra, rj, rs, rn, sp, m, n, &sc->err, u, low);
        else
            correct_lane<6>(st, idx, ra, rj, rs, rn, sp, m, n, &sc->err, u, low);
    }
    if (!min_pass) return;
    // Next block time: min over the new tend of the particles corrected here and
    // over every particle whose tend differs from the block time.  A particle of
    // the block read while another CTA corrects it shows either its old tend
    // (== block time: skipped, its new value is in that CTA's minimum) or its new
    // one (final): no ordering between CTAs is needed.
    const long long tb = __double_as_longlong(*((volatile double *)&sc->t_cur));
    const volatile long long *bits = reinterpret_cast<const volatile long long *>(st.tend);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const long long v = bits[i];
        if (v != tb) low = min(low, v);
    }
    low = block_min_ll(low, sh);
    if (threadIdx.x == 0 && low != LLONG_MAX) atomicMin((long long *)&sc->tnext_bits, low);
}


// ------------------------------------------------------------------------
// Energy: Sect. 2 softened potential, W = -1/2 sum_i m_i sum_{j != i} m_j /
// sqrt(r^2 + eps^2), kinetic 1/2 sum m v^2.  Per-i potentials over j-chunks,
// then ordered sums.
// ------------------------------------------------------------------------
constexpr int kPotThreads = 128;

template <bool MIXED>
__global__ void __launch_bounds__(kPotThreads) k_potential(const double *xe, const double *mass, int64_t n,
                                                            int64_t jchunk, double eps2, double *phi_part)
{
    __shared__ double sx[kPotThreads], sy[kPotThreads], sz[kPotThreads], sm[kPotThreads];
    __shared__ float fh[3][kPotThreads], fl[3][kPotThreads], fm[kPotThreads];
    const int64_t i = blockIdx.x * (int64_t)kPotThreads + threadIdx.x;
    const int64_t ic = i < n ? i : n - 1;
    const int64_t j0 = blockIdx.y * jchunk;
    const int64_t j1 = (j0 + jchunk < n) ? j0 + jchunk : n;
    double xi[3] = {xe[3 * ic], xe[3 * ic + 1], xe[3 * ic + 2]};
    float xih[3], xil[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xih[k] = __double2float_rn(xi[k]);
        xil[k] = __double2float_rn(xi[k] - (double)xih[k]);
    }
    double phi = 0.0;
    float hi = 0.f, lo = 0.f;
    const float eps2f = (float)eps2;
    for (int64_t jb = j0; jb < j1; jb += kPotThreads) {
        const int64_t j = jb + threadIdx.x;
        __syncthreads();
        if (j < j1) {
            if (MIXED) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double x = xe[3 * j + k];
                    fh[k][threadIdx.x] = __double2float_rn(x);
                    fl[k][threadIdx.x] = __double2float_rn(x - (double)fh[k][threadIdx.x]);
                }
                fm[threadIdx.x] = __double2float_rn(mass[j]);
            } else {
                sx[threadIdx.x] = xe[3 * j];
                sy[threadIdx.x] = xe[3 * j + 1];
                sz[threadIdx.x] = xe[3 * j + 2];
                sm[threadIdx.x] = mass[j];
            }
        }
        __syncthreads();
        const int cnt = (int)((j1 - jb) < kPotThreads ? (j1 - jb) : kPotThreads);
        if (MIXED) {
            float ch = 0.f;
            for (int u = 0; u < cnt; ++u) {
                const float dx = (fh[0][u] - xih[0]) + (fl[0][u] - xil[0]);
                const float dy = (fh[1][u] - xih[1]) + (fl[1][u] - xil[1]);
                const float dz = (fh[2][u] - xih[2]) + (fl[2][u] - xil[2]);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2f)));
                float r = rsqrt_approx(r2);
                r = r * fmaf(-0.5f * r2, r * r, 1.5f);           // one Newton step
                ch += (jb + u == i) ? 0.f : fm[u] * r;
            }
            const float y = ch - lo;
            const float tt = hi + y;
            lo = (tt - hi) - y;
            hi = tt;
        } else {
            for (int u = 0; u < cnt; ++u) {
                const double dx = sx[u] - xi[0], dy = sy[u] - xi[1], dz = sz[u] - xi[2];
                const double r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
                phi += (jb + u == i) ? 0.0 : sm[u] * rsqrt(r2);
            }
        }
    }
    if (MIXED) phi = (double)hi - (double)lo;
    if (i < n) phi_part[blockIdx.y * n + i] = phi;
}

// Independent clusters: phi_i sums over the other particles of i's own cluster
// only (FP64 pairs, read from global memory; cluster sizes are modest).
__global__ void k_potential_clusters(const double *xe, const double *mass, const int32_t *cl_of,
                                     const int64_t *cl_off, int64_t n, double eps2, double *phi)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cl_of[i];
        const double xi = xe[3 * i], yi = xe[3 * i + 1], zi = xe[3 * i + 2];
        double s = 0.0;
        for (int64_t j = cl_off[c]; j < cl_off[c + 1]; ++j) {
            const double dx = xe[3 * j] - xi, dy = xe[3 * j + 1] - yi, dz = xe[3 * j + 2] - zi;
            const double r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
            s += (j == i) ? 0.0 : mass[j] * rsqrt(r2);
        }
        phi[i] = s;
    }
}

__global__ void k_energy_sum(const double *mass, const double *ve, const double *phi_part, int64_t n, int nsplit,
                             double *part2)
{
    __shared__ double shk[32], shw[32];
    double k = 0.0, w = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double phi = 0.0;
        for (int s = 0; s < nsplit; ++s) phi += phi_part[s * n + i];
        const double vx = ve[3 * i], vy = ve[3 * i + 1], vz = ve[3 * i + 2];
        k += 0.5 * mass[i] * (vx * vx + vy * vy + vz * vz);
        w += mass[i] * phi;
    }
    for (int off = 16; off > 0; off >>= 1) {
        k += __shfl_xor_sync(0xffffffffu, k, off);
        w += __shfl_xor_sync(0xffffffffu, w, off);
    }
    const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        shk[wp] = k;
        shw[wp] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sk = 0.0, sw = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            sk += shk[q];
            sw += shw[q];
        }
        part2[2 * blockIdx.x] = sk;
        part2[2 * blockIdx.x + 1] = sw;
    }
}

__global__ void k_energy_final(const double *part2, int g, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double k = 0.0, w = 0.0;
        for (int c = 0; c < g; ++c) {
            k += part2[2 * c];
            w += part2[2 * c + 1];
        }
        out[0] = k;
        out[1] = -0.5 * w;
    }
}

// Total angular momentum sum_i m_i r_i x v_i of the predicted system (the
// conservation check of Sect. 5.1): per-CTA FP64 partial sums in a fixed
// order, then one thread adds the g partials in CTA order (deterministic).
__global__ void k_angmom_sum(const double *mass, const double *xe, const double *ve, int64_t n, double *part3)
{
    __shared__ double sh[3][32];
    double L[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *r = xe + 3 * i, *u = ve + 3 * i;
        L[0] += mass[i] * (r[1] * u[2] - r[2] * u[1]);
        L[1] += mass[i] * (r[2] * u[0] - r[0] * u[2]);
        L[2] += mass[i] * (r[0] * u[1] - r[1] * u[0]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) L[c] += __shfl_xor_sync(0xffffffffu, L[c], off);
    const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int c = 0; c < 3; ++c) sh[c][wp] = L[c];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[c][k];
            part3[3 * blockIdx.x + c] = t;
        }
}

__global__ void k_angmom_final(const double *part3, int g, double *out3)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            double t = 0.0;
            for (int k = 0; k < g; ++k) t += part3[3 * k + c];
            out3[c] = t;
        }
}

// ------------------------------------------------------------------------
// Validation (flags, never traps).
// ------------------------------------------------------------------------
__device__ __forceinline__ bool is_pow2(double x)
{
    int e;
    return x > 0.0 && isfinite(x) && frexp(x, &e) == 0.5;
}

// |x| <= lim (false for NaN and infinities).
__device__ __forceinline__ bool within(double x, double lim) { return fabs(x) <= lim; }

__global__ void k_validate_init(const double *mass, const double *x, const double *v, int64_t n, ValueLimits lim,
                                int32_t *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        bool ok = isfinite(mass[i]) && mass[i] > 0.0;
        for (int k = 0; k < 3; ++k) ok = ok && within(x[3 * i + k], lim.pos) && within(v[3 * i + k], lim.deriv);
        if (!ok) atomicOr(flag, ERR_VALUE);
    }
}

__global__ void k_validate_state(const State st, int64_t n, double dt_min, double dt_max, ValueLimits lim,
                                 int32_t *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        bool ok = isfinite(st.mass[i]) && st.mass[i] > 0.0 && isfinite(st.t[i]) && st.t[i] >= 0.0;
        for (int k = 0; k < 3; ++k) {
            const int64_t q = 3 * i + k;
            ok = ok && within(st.x[q], lim.pos) && within(st.v[q], lim.deriv) && within(st.a[q], lim.deriv) &&
                 within(st.j[q], lim.deriv) && within(st.s[q], lim.deriv) && within(st.c[q], lim.deriv);
        }
        const double dt = st.dt[i];
        ok = ok && is_pow2(dt) && dt >= dt_min && dt <= dt_max && fmod(st.t[i], dt) == 0.0;
        if (!ok) atomicOr(flag, ERR_VALUE);
    }
}

__global__ void k_validate_idx(const int32_t *idx, int64_t m, int64_t n, int32_t *flag)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = idx[q];
        bool ok = i >= 0 && (int64_t)i < n;
        if (q > 0) ok = ok && idx[q - 1] < i;
        if (!ok) atomicOr(flag, ERR_BADIDX);
    }
}

// hg_correct preconditions: same list as the evaluation (when given) and every
// listed particle due exactly at the prediction time.
__global__ void k_check_correct(const State st, const int32_t *given, const int32_t *cur, int64_t m, int64_t n,
                                double t_pred, int32_t *flag)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = cur[q];
        bool ok = (given == nullptr) || (given[q] == i);
        ok = ok && i >= 0 && (int64_t)i < n && (st.t[i] + st.dt[i] == t_pred);
        if (!ok) atomicOr(flag, ERR_STATE);
    }
}

// ------------------------------------------------------------------------
// Work list of one evaluation over independent clusters (one CTA).  For each
// cluster: its range of the (ascending) active list by binary search, threads
// per i-particle from its active count, j-chunks of tps tiles over its own
// records; tps is common: the largest power of two up to 64 that still gives
// at least two items per resident CTA (smaller tps only if the partial-sum
// capacity allows).  Exclusive scans give each cluster's first work item and
// first partial-sum row.
// ------------------------------------------------------------------------
constexpr int kPlanThreads = 1024;
constexpr int kTpsCand = 7;   // tps = 1, 2, ..., 64

__device__ void block_exscan_i64(int64_t v, int64_t *sh, int64_t &excl, int64_t &total)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += u;
    }
    __syncthreads();
    if (l == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int64_t x = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0;
        int64_t xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, xi, o);
            if (l >= o) xi += u;
        }
        sh[l] = xi - x;
        if (l == 31) sh[32] = xi;
    }
    __syncthreads();
    excl = sh[w] + incl - v;
    total = sh[32];
    __syncthreads();
}

// Threads per i-particle of a cluster with mc active particles: the largest
// power of two that still fills one CTA (ipt particles per thread), times 2^shift.
__device__ __forceinline__ int batch_tpi(int64_t mc, int ipt, int shift)
{
    int tpi = 1;
    const int64_t want = (int64_t)kEvalThreads * ipt / mc;
    while (tpi * 2 <= want && tpi < kMaxTPI) tpi *= 2;
    if (shift > 0 && tpi < kMaxTPI) tpi *= 2;
    if (shift < 0 && tpi > 1) tpi /= 2;
    return tpi;
}

__global__ void __launch_bounds__(kPlanThreads) k_batch_plan(const int32_t *idx, const int64_t *m_dev, int64_t m_host,
                                                             BatchView bv, PlanParams q, DevScalars *count)
{
    __shared__ int64_t sh[33];
    __shared__ int64_t s_tps;
    const int64_t m = m_dev ? *m_dev : m_host;
    if (m <= 0) return;
    const int nc = bv.nc;
    const int tj = q.tj, ipt = q.i_per_thread, grid = q.grid;
    const int64_t pcap = q.pcap;
    const BatchKnobs kn = batch_knobs(m, q);
    for (int c = threadIdx.x; c <= nc; c += blockDim.x) {
        if (c == nc) {
            bv.a_off[nc] = m;
            continue;
        }
        const int64_t key = bv.cl_off[c];
        int64_t lo = 0, hi = m;   // first position with idx >= key
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (idx[mid] < key) lo = mid + 1; else hi = mid;
        }
        bv.a_off[c] = lo;
    }
    __syncthreads();
    // This thread's clusters [c0, c1): active counts and tiles.
    const int per = (nc + (int)blockDim.x - 1) / (int)blockDim.x;
    const int c0 = threadIdx.x * per, c1 = (c0 + per < nc) ? c0 + per : nc;
    int64_t items[kTpsCand], parts[kTpsCand];
    for (int k = 0; k < kTpsCand; ++k) items[k] = parts[k] = 0;
    for (int c = c0; c < c1; ++c) {
        const int64_t mc = bv.a_off[c + 1] - bv.a_off[c];
        if (mc == 0) continue;
        const int tpi = batch_tpi(mc, ipt, kn.tpi_shift);
        const int64_t ti = kEvalThreads / tpi * ipt;
        const int64_t nit = (mc + ti - 1) / ti;
        const int64_t ntc = (bv.rec_off[c + 1] - bv.rec_off[c]) / tj;
        for (int k = 0; k < kTpsCand; ++k) {
            const int64_t b = (ntc + (1 << k) - 1) >> k;
            items[k] += nit * b;
            parts[k] += b * mc;
        }
    }
    for (int k = 0; k < kTpsCand; ++k) {
        int64_t e, t;
        block_exscan_i64(items[k], sh, e, t);
        items[k] = t;
        block_exscan_i64(parts[k], sh, e, t);
        parts[k] = t;
    }
    if (threadIdx.x == 0) {
        int pick = -1;
        for (int k = kTpsCand - 1; k >= 0 && pick < 0; --k)
            if (parts[k] <= pcap && items[k] >= ((int64_t)grid << kn.w_log)) pick = k;
        for (int k = 0; k < kTpsCand && pick < 0; ++k)
            if (parts[k] <= pcap) pick = k;
        if (pick < 0) pick = kTpsCand - 1;
        s_tps = (int64_t)1 << pick;
        *bv.tps = s_tps;
    }
    __syncthreads();
    const int64_t tps = s_tps;
    int64_t my_items = 0, my_parts = 0;
    for (int c = c0; c < c1; ++c) {
        const int64_t mc = bv.a_off[c + 1] - bv.a_off[c];
        const int tpi = mc > 0 ? batch_tpi(mc, ipt, kn.tpi_shift) : 1;
        const int64_t ti = kEvalThreads / tpi * ipt;
        const int64_t nit = (mc + ti - 1) / ti;
        const int64_t ntc = (bv.rec_off[c + 1] - bv.rec_off[c]) / tj;
        const int64_t b = (ntc + tps - 1) / tps;
        bv.tpi_c[c] = tpi;
        bv.b_c[c] = (int32_t)b;
        my_items += nit * b;
        my_parts += b * mc;
    }
    int64_t ie, it, pe, pt, we, wt, my_pred = 0;
    for (int c = c0; c < c1; ++c)
        if (bv.a_off[c + 1] > bv.a_off[c]) my_pred += bv.cl_off[c + 1] - bv.cl_off[c];
    block_exscan_i64(my_pred, sh, we, wt);
    for (int c = c0; c < c1; ++c) {
        bv.pred_off[c] = we;
        if (bv.a_off[c + 1] > bv.a_off[c]) we += bv.cl_off[c + 1] - bv.cl_off[c];
    }
    if (threadIdx.x == 0) bv.pred_off[nc] = wt;
    block_exscan_i64(my_items, sh, ie, it);
    block_exscan_i64(my_parts, sh, pe, pt);
    if (count) {   // pair evaluations of this block step: sum over clusters of m_c N_c
        int64_t my_pairs = 0;
        for (int c = c0; c < c1; ++c)
            my_pairs += (bv.a_off[c + 1] - bv.a_off[c]) * (bv.cl_off[c + 1] - bv.cl_off[c]);
        int64_t e, tot;
        block_exscan_i64(my_pairs, sh, e, tot);
        if (threadIdx.x == 0) count->interactions += tot;
    }
    for (int c = c0; c < c1; ++c) {
        const int64_t mc = bv.a_off[c + 1] - bv.a_off[c];
        const int64_t ti = kEvalThreads / bv.tpi_c[c] * ipt;
        const int64_t nit = (mc + ti - 1) / ti;
        bv.item_off[c] = ie;
        bv.part_off[c] = pe;
        ie += nit * bv.b_c[c];
        pe += (int64_t)bv.b_c[c] * mc;
    }
    if (threadIdx.x == 0) {
        bv.item_off[nc] = it;
        bv.part_off[nc] = pt;
    }
}

// Zero-mass padding records far away in every slot (before the first prediction
// of a cluster context, whose particles do not cover all record slots).
template <bool MIXED>
__global__ void k_pad_records(Records rec, int64_t npad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (MIXED) {
            const float far = (float)kPadCoord;
            store_mixed_record(rec, i, MixedRecord{far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f});
        } else {
            static_cast<double2 *>(rec.p[0])[i] = make_double2(kPadCoord, kPadCoord);
            static_cast<double2 *>(rec.p[1])[i] = make_double2(kPadCoord, 0.0);
            static_cast<double2 *>(rec.p[2])[i] = make_double2(0.0, 0.0);
            static_cast<double2 *>(rec.p[3])[i] = make_double2(0.0, 0.0);
            static_cast<double2 *>(rec.p[4])[i] = make_double2(0.0, 0.0);
        }
    }
}

// tend = t + dt for every particle (after the state is replaced).
__global__ void k_tend(State st, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        st.tend[i] = st.t[i] + st.dt[i];
}

inline int grid_for(int64_t work, int threads, int cap)
{
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
int nb_grid(int64_t n) { return (int)((n + kNBChunk - 1) / kNBChunk); }

cudaError_t launch_next_block(const State &st, int64_t n, double *part, int32_t *cnt, int32_t *off, int32_t *idx,
                              DevScalars *sc, int count_step, const PlanParams &pq, cudaStream_t s)
{
    const int g = nb_grid(n);
    long long *bits = reinterpret_cast<long long *>(part);
    k_nb_min<<<g, kNBThreads, 0, s>>>(st.tend, n, kNBChunk, bits, g, sc);
    k_nb_count<<<g, kNBThreads, 0, s>>>(st.tend, n, kNBChunk, cnt, off, g, sc, count_step, pq);
    k_nb_scatter<<<g, kNBThreads, 0, s>>>(st.tend, n, kNBChunk, off, idx, sc);
    return cudaGetLastError();
}

cudaError_t launch_next_min(const State &st, int64_t n, double *part, DevScalars *sc, cudaStream_t s)
{
    const int g = nb_grid(n);
    k_nb_min<<<g, kNBThreads, 0, s>>>(st.tend, n, kNBChunk, reinterpret_cast<long long *>(part), g, sc);
    return cudaGetLastError();
}

cudaError_t launch_tend(const State &st, int64_t n, cudaStream_t s)
{
    k_tend<<<grid_for(n, 256, 4096), 256, 0, s>>>(st, n);
    return cudaGetLastError();
}

cudaError_t launch_predict(bool mixed, const State &st, const Records &rec, int64_t n, int64_t npad,
                           const double *t_dev, double t_host, const int64_t *m_dev, const int32_t *rmap,
                           cudaStream_t s)
{
    const int g = grid_for(rmap ? n : npad, 64, 1 << 20);   // small CTAs: even spread of the FP64 work
    if (mixed)
        k_predict<true><<<g, 64, 0, s>>>(st, rec, n, npad, t_dev, t_host, m_dev, rmap);
    else
        k_predict<false><<<g, 64, 0, s>>>(st, rec, n, npad, t_dev, t_host, m_dev, rmap);
    return cudaGetLastError();
}

cudaError_t launch_predict_select(bool mixed, const State &st, const Records &rec, int64_t n, int64_t npad,
                                  int32_t *idx, DevScalars *sc, int count_step, const PlanParams &pq, int max_grid,
                                  cudaStream_t s)
{
    // Persistent grid: every CTA takes one atomic on the arrival counter, and
    // at N = 2^20 sixteen thousand of them on one address cost more than the
    // prediction itself.
    const int g = grid_for(npad, 256, max_grid);
    if (mixed)
        k_predict_select<true><<<g, 256, 0, s>>>(st, rec, n, npad, idx, sc, count_step, pq);
    else
        k_predict_select<false><<<g, 256, 0, s>>>(st, rec, n, npad, idx, sc, count_step, pq);
    return cudaGetLastError();
}

cudaError_t launch_predict_clusters(bool mixed, const State &st, const Records &rec, int64_t n, const BatchView &bv,
                                    const double *t_dev, const int64_t *m_dev, cudaStream_t s)
{
    const int g = grid_for(n, 64, 1 << 20);
    if (mixed)
        k_predict_clusters<true><<<g, 64, 0, s>>>(st, rec, n, bv, t_dev, m_dev);
    else
        k_predict_clusters<false><<<g, 64, 0, s>>>(st, rec, n, bv, t_dev, m_dev);
    return cudaGetLastError();
}

cudaError_t launch_pad_records(bool mixed, const Records &rec, int64_t npad, cudaStream_t s)
{
    if (mixed)
        k_pad_records<true><<<grid_for(npad, 256, 1 << 20), 256, 0, s>>>(rec, npad);
    else
        k_pad_records<false><<<grid_for(npad, 256, 1 << 20), 256, 0, s>>>(rec, npad);
    return cudaGetLastError();
}

cudaError_t launch_batch_plan(const int32_t *idx, const int64_t *m_dev, int64_t m_host, const BatchView &bv,
                              const PlanParams &q, DevScalars *count, cudaStream_t s)
{
    k_batch_plan<<<1, kPlanThreads, 0, s>>>(idx, m_dev, m_host, bv, q, count);
    return cudaGetLastError();
}

cudaError_t launch_start(const State &st, int64_t n, const double *ra, const double *rj, const double *rs,
                         const StepParams &sp, cudaStream_t s)
{
    k_start<<<grid_for(n, 256, 1 << 20), 256, 0, s>>>(st, n, ra, rj, rs, sp);
    return cudaGetLastError();
}

cudaError_t launch_correct(const State &st, const int32_t *idx, const int64_t *m_dev, int64_t m_host, int64_t n,
                           const double *ra, const double *rj, const double *rs, const double *rn,
                           const StepParams &sp, DevScalars *sc, int min_pass, int grid, cudaStream_t s)
{
    k_correct<<<grid, 128, 0, s>>>(st, idx, m_dev, m_host, ra, rj, rs, rn, sp, sc, n, min_pass);
    return cudaGetLastError();
}

int energy_splits(int64_t n, int num_sms)
{
    const int64_t itiles = (n + kPotThreads - 1) / kPotThreads;
    int64_t b = (4 * (int64_t)num_sms + itiles - 1) / itiles;
    const int64_t jt = (n + kPotThreads - 1) / kPotThreads;
    if (b > jt) b = jt;
    if (b > 64) b = 64;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_energy(bool mixed, const State &st, int64_t n, double t, double eps2, double *xe, double *ve,
                          double *phi_part, int nsplit, double *part2, int g2, double *out2, const BatchView &bv,
                          cudaStream_t s)
{
    k_predict_xv<<<grid_for(n, 256, 1 << 20), 256, 0, s>>>(st, n, t, xe, ve);
    int64_t jchunk = (n + nsplit - 1) / nsplit;
    jchunk = (jchunk + kPotThreads - 1) / kPotThreads * kPotThreads;
    dim3 grid((unsigned)((n + kPotThreads - 1) / kPotThreads), (unsigned)nsplit);
    if (bv.nc > 0) {
        k_potential_clusters<<<grid_for(n, 128, 1 << 20), 128, 0, s>>>(xe, st.mass, bv.cl_of, bv.cl_off, n, eps2,
                                                                        phi_part);
        nsplit = 1;
    } else if (mixed) {
        k_potential<true><<<grid, kPotThreads, 0, s>>>(xe, st.mass, n, jchunk, eps2, phi_part);
    } else {
        k_potential<false><<<grid, kPotThreads, 0, s>>>(xe, st.mass, n, jchunk, eps2, phi_part);
    }
    k_energy_sum<<<g2, 256, 0, s>>>(st.mass, ve, phi_part, n, nsplit, part2);
    k_energy_final<<<1, 32, 0, s>>>(part2, g2, out2);
    return cudaGetLastError();
}

cudaError_t launch_angular_momentum(const State &st, int64_t n, double t, double *xe, double *ve, double *part3,
                                    int g, double *out3, cudaStream_t s)
{
    k_predict_xv<<<grid_for(n, 256, 1 << 20), 256, 0, s>>>(st, n, t, xe, ve);
    k_angmom_sum<<<g, 256, 0, s>>>(st.mass, xe, ve, n, part3);
    k_angmom_final<<<1, 32, 0, s>>>(part3, g, out3);
    return cudaGetLastError();
}

cudaError_t launch_validate_init(const double *mass, const double *x, const double *v, int64_t n,
                                 const ValueLimits &lim, int32_t *flag, cudaStream_t s)
{
    k_validate_init<<<grid_for(n, 256, 4096), 256, 0, s>>>(mass, x, v, n, lim, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate_state(const State &st, int64_t n, double dt_min, double dt_max, const ValueLimits &lim,
                                  int32_t *flag, cudaStream_t s)
{
    k_validate_state<<<grid_for(n, 256, 4096), 256, 0, s>>>(st, n, dt_min, dt_max, lim, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate_idx(const int32_t *idx, int64_t m, int64_t n, int32_t *flag, cudaStream_t s)
{
    k_validate_idx<<<grid_for(m, 256, 4096), 256, 0, s>>>(idx, m, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_check_correct(const State &st, const int32_t *given, const int32_t *cur, int64_t m, int64_t n,
                                 double t_pred, int32_t *flag, cudaStream_t s)
{
    k_check_correct<<<grid_for(m, 256, 4096), 256, 0, s>>>(st, given, cur, m, n, t_pred, flag);
    return cudaGetLastError();
}

}  // namespace hg
