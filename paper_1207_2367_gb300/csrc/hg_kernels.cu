// hg_kernels.cu -- the FP64 parts of a block step (next-block selection,
// predictor, corrector with the time-step update), start-up, energy and
// input validation.  Sect. 3 of the HiGPUs paper; Table 1 sections 1, 2, 8.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hg_kernels.cuh"
#include "hg_step_dev.cuh"

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
    if (take) plan_on_block(tot, pq, reinterpret_cast<Plan *>(sc->plan));   // uniform: every thread of the CTA
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
    predict_select_pass<MIXED>(st, rec, n, npad, idx, sc, tn, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                               (int64_t)gridDim.x * blockDim.x);
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
    plan_on_block(m > 0 ? m : 1, pq, reinterpret_cast<Plan *>(sc->plan));
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

__global__ void __launch_bounds__(128) k_correct(State st, const int32_t *idx, const int64_t *m_dev, int64_t m_host,
                                                 const double *ra, const double *rj, const double *rs,
                                                 const double *rn, StepParams sp, DevScalars *sc, int64_t n,
                                                 int min_pass)
{
    __shared__ long long sh[32];
    const int64_t m = m_dev ? *m_dev : m_host;
    if (m <= 0) return;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, G = (int64_t)gridDim.x * blockDim.x;
    long long low = LLONG_MAX;
    if (min_pass) low = scan_min_pass(st, n, __double_as_longlong(*((volatile double *)&sc->t_cur)), g, G);
    correct_pass(st, idx, m, n, ra, rj, rs, rn, sp, &sc->err, g >> 5, G >> 5, low);
    if (min_pass) publish_min(sc, low, sh);
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
        bool ok = isfinite(mass[i]) && mass[i] > 0.0 && mass[i] <= lim.mass;
        for (int k = 0; k < 3; ++k) ok = ok && within(x[3 * i + k], lim.pos) && within(v[3 * i + k], lim.deriv);
        if (!ok) atomicOr(flag, ERR_VALUE);
    }
}

__global__ void k_validate_state(const State st, int64_t n, double dt_min, double dt_max, ValueLimits lim,
                                 int32_t *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        bool ok = isfinite(st.mass[i]) && st.mass[i] > 0.0 && st.mass[i] <= lim.mass && isfinite(st.t[i]) &&
                  st.t[i] >= 0.0;
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
// The fields derived from the state: tend = t + dt and (mixed) the FP32 copies.
__global__ void k_tend(State st, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        st.tend[i] = st.t[i] + st.dt[i];
        if (st.f32) store_f32(st, i);
    }
}

__global__ void k_f32(State st, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        store_f32(st, i);
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

cudaError_t launch_f32(const State &st, int64_t n, cudaStream_t s)
{
    if (!st.f32) return cudaSuccess;
    k_f32<<<grid_for(n, 256, 4096), 256, 0, s>>>(st, n);
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
