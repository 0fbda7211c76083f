// hg_step_dev.cuh -- device code of the block step (hg_kernels.cu): the
// evaluation planner on one CTA, CTA reductions and arrival counts, the FP64
// predictor (Sect. 3 item 1), the corrector with the Hermite interpolation and
// the step criterion (Sect. 3 item 3, criterion equations, power-of-two
// blocks), and the passes of a graph-replayed block step.
#pragma once

#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "hg_kernels.cuh"

namespace hg {
namespace {

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
// Thread 0 writes *out (global or shared memory).
__device__ void plan_on_block(int64_t m, const PlanParams &q, Plan *out)
{
    __shared__ int64_t s_cost[32];
    __shared__ int s_cand[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    Plan p;
    const int tc = q.tuned[tune_bucket(m)];
    if (tc >= 0 && plan_candidate(m, q, tc, p) >= 0) {   // measured choice
        if (threadIdx.x == 0) *out = p;
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
        *out = p;
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

// ------------------------------------------------------------------------
// Sect. 3 item 1: Taylor predictor through crackle, FP64, h = t - t_j.
// ------------------------------------------------------------------------
struct Pred {
    double x[3], v[3], a[3];
};

__device__ __forceinline__ Pred predict_one(const State &st, int64_t i, double tt)
{
    Pred p;
    const double h = tt - __ldcg(st.t + i);
    const double h2 = h * h * 0.5;              // h^2/2
    const double h3 = h2 * h * (1.0 / 3.0);     // h^3/6
    const double h4 = h3 * h * 0.25;            // h^4/24
    const double h5 = h4 * h * 0.2;             // h^5/120
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t q = 3 * i + k;
        const double x = __ldcg(st.x + q), v = __ldcg(st.v + q), a = __ldcg(st.a + q), j = __ldcg(st.j + q),
                     s = __ldcg(st.s + q), c = __ldcg(st.c + q);
        p.x[k] = x + fma(h, v, fma(h2, a, fma(h3, j, fma(h4, s, h5 * c))));
        p.v[k] = v + fma(h, a, fma(h2, j, fma(h3, s, h4 * c)));
        p.a[k] = a + fma(h, j, fma(h2, s, h3 * c));
    }
    return p;
}

// The 16 FP32 values of particle i (mixed contexts), from its FP64 fields.
__device__ __forceinline__ void store_f32(const State &st, int64_t i)
{
    float f[16];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t q = 3 * i + k;
        f[kF32V + k] = d2f(__ldcg(st.v + q));
        f[kF32A + k] = d2f(__ldcg(st.a + q));
        f[kF32J + k] = d2f(__ldcg(st.j + q));
        f[kF32S + k] = d2f(__ldcg(st.s + q));
        f[kF32C + k] = d2f(__ldcg(st.c + q));
    }
    f[kF32M] = d2f(__ldcg(st.mass + i));
#pragma unroll
    for (int w = 0; w < 4; ++w) st.f32[4 * i + w] = make_float4(f[4 * w], f[4 * w + 1], f[4 * w + 2], f[4 * w + 3]);
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
                // component (at 64 cycles per warp instruction the FP64 unit
                // shares this kernel's limit with DRAM on GB300).
                // Velocities and accelerations feed only the FP32 pair
                // arithmetic: FP32 Horner series from the rounded derivatives.
                // The FP32 inputs come rounded already (st.f32): the same
                // values as d2f of the FP64 fields, without the conversions.
                const double h = tt - __ldcg(st.t + i);
                const float hf = d2f(h);
                float f[16];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const float4 u = __ldcg(st.f32 + 4 * i + w);
                    f[4 * w] = u.x;
                    f[4 * w + 1] = u.y;
                    f[4 * w + 2] = u.z;
                    f[4 * w + 3] = u.w;
                }
                float hi[3], lo[3], vp[3], ap[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int64_t q = 3 * i + k;
                    const double x = __ldcg(st.x + q), v = __ldcg(st.v + q);
                    const float vf = f[kF32V + k], af = f[kF32A + k], jf = f[kF32J + k], sf = f[kF32S + k],
                                cf = f[kF32C + k];
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
                v = MixedRecord{hi[0], hi[1], hi[2], f[kF32M], lo[0], lo[1], lo[2], ap[0],
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
                q1 = make_double2(p.x[2], __ldcg(st.mass + i));
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
// Component k of one particle's fields at the start of its step, loaded in one
// round trip with its t and dt.
struct CorrIn {
    double x0, v0, a0, j0, s0;
};

__device__ __forceinline__ void correct_component(const State &st, int64_t i, int k, double h, int e, bool pow2,
                                                  const CorrIn &in, double a1, double j1, double s1, double &c3,
                                                  double &c4, double &c5, double &Ak)
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
    const double x0 = in.x0, v0 = in.v0, a0 = in.a0, j0 = in.j0, s0 = in.s0;
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
    if (st.f32) {
        float *f = reinterpret_cast<float *>(st.f32 + 4 * i);
        f[kF32V + k] = d2f(v1);
        f[kF32A + k] = d2f(a1);
        f[kF32J + k] = d2f(j1);
        f[kF32S + k] = d2f(s1);
        f[kF32C + k] = d2f(c3);
    }
}

// 4th-order scheme, component k of particle i (the two-point Hermite corrector
// and the cubic interpolant through a and jerk at both ends): corrected v and r,
// new a and jerk (snap and crackle stored as zero: the predictor ends at jerk),
// and snap and crackle at the step's end for the p = 4 criterion.  h = 2^e:
// h^2/12 = 2^(2e) fl(1/12) and the reciprocal powers are exact scalings.
__device__ __forceinline__ void correct4_component(const State &st, int64_t i, int k, double h, int e, bool pow2,
                                                   const CorrIn &in, double a1, double j1, double &s1, double &c1,
                                                   double &Ak)
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
    const double x0 = in.x0, v0 = in.v0, a0 = in.a0, j0 = in.j0;
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
    if (st.f32) {
        float *f = reinterpret_cast<float *>(st.f32 + 4 * i);
        f[kF32V + k] = d2f(v1);
        f[kF32A + k] = d2f(a1);
        f[kF32J + k] = d2f(j1);
        f[kF32S + k] = 0.f;
        f[kF32C + k] = 0.f;
    }
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

// New time t0 + h and p = 6 step of particle i from d = a^(0..5) at the step's end.
// A: the acceleration change left after a0 + j0 h + s0 h^2/2 (a0 + j0 h for
// p = 4).  Below the noise floor of the evaluation, sp.noise_rel times the
// noise scale (sum_j m_j / r_ij^2 where the evaluation provides it, else |a1|;
// compared as squares), the interpolated derivatives are noise and the
// criterion may not shrink the step.
template <int P>
__device__ __forceinline__ double finish_step(const State &st, int64_t i, double t0, double h, int e, bool pow2,
                                              const double (*d)[3], const double *A, double scale2,
                                              const StepParams &sp, bool store)
{
    const double t1 = t0 + h;
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
    // What is indexed by the list position q is loaded at once, then the
    // particle's own fields in one more round trip: the chain of dependent
    // loads ahead of the arithmetic is two deep.
    int32_t iq = 0;
    double dk[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, rnq = 0.0;
    if (act) {
        iq = __ldcg(idx + q);
        dk[0] = __ldcg(ra + 3 * q + k);
        dk[1] = __ldcg(rj + 3 * q + k);
        if (P == 6) dk[2] = __ldcg(rs + 3 * q + k);
        if (rn) rnq = __ldcg(rn + q);
    }
    if (act && !in_bounds(iq >= 0 && (int64_t)iq < n, err)) act = false;
    double Ak = 0.0, h = 1.0, t0 = 0.0;
    int64_t i = 0;
    int e = 0;
    bool pow2 = false;
    if (act) {
        i = iq;
        const int64_t qk = 3 * i + k;
        h = __ldcg(st.dt + i);
        t0 = __ldcg(st.t + i);
        CorrIn in;
        in.x0 = __ldcg(st.x + qk);
        in.v0 = __ldcg(st.v + qk);
        in.a0 = __ldcg(st.a + qk);
        in.j0 = __ldcg(st.j + qk);
        in.s0 = P == 6 ? __ldcg(st.s + qk) : 0.0;
        pow2 = pow2_exponent(h, e);
        if (P == 4)
            correct4_component(st, i, k, h, e, pow2, in, dk[0], dk[1], dk[2], dk[3], Ak);
        else
            correct_component(st, i, k, h, e, pow2, in, dk[0], dk[1], dk[2], dk[3], dk[4], dk[5], Ak);
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
        const double scale2 = rn ? rnq * rnq : sq3(d[0]);
        low = min(low, __double_as_longlong(finish_step<P>(st, i, t0, h, e, pow2, d, A, scale2, sp, k == 0)));
    }
}


// ------------------------------------------------------------------------
// Passes of a graph-replayed block step of one system, taken by global thread
// g of G (grid-stride).  State, lists and results are read through L2
// (__ldcg) or volatile, never through the read-only path: a pass must see what
// other CTAs wrote earlier, whatever kernel it runs in.
// ------------------------------------------------------------------------

// Table 1 sections 1-2 in one pass: predict every record to t_next (bit
// pattern tn) and append each particle with tend_i == t_next to idx, one
// atomic on sc->slot per warp (the list order is arbitrary: a particle's sums
// do not depend on its position).  Whole warps take part (the ballot).
template <bool MIXED>
__device__ void predict_select_pass(const State &st, const Records &rec, int64_t n, int64_t npad, int32_t *idx,
                                    DevScalars *sc, long long tn, int64_t g0, int64_t G)
{
    const double t_next = __longlong_as_double(tn);
    const long long *bits = reinterpret_cast<const long long *>(st.tend);
    const int l = threadIdx.x & 31;
    for (int64_t base = g0 - l; base < npad; base += G) {
        const int64_t i = base + l;
        if (i < npad) predict_record<MIXED>(st, rec, i, n, i, t_next);
        const bool due = i < n && __ldcg(bits + i) == tn;
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
}

// Table 1 section 8: correct the m listed particles and take their new steps,
// three lanes per particle in units of kCorrUnit particles per warp; warp w of
// W takes units w, w + W, ...  low receives the minimum of their new tend.
__device__ void correct_pass(const State &st, const int32_t *idx, int64_t m, int64_t n, const double *ra,
                             const double *rj, const double *rs, const double *rn, const StepParams &sp, int32_t *err,
                             int64_t w, int64_t W, long long &low)
{
    const int64_t units = (m + kCorrUnit - 1) / kCorrUnit;
    for (int64_t u = w; u < units; u += W) {   // warp-uniform
        if (sp.order == 4)
            correct_lane<4>(st, idx, ra, rj, rs, rn, sp, m, n, err, u, low);
        else
            correct_lane<6>(st, idx, ra, rj, rs, rn, sp, m, n, err, u, low);
    }
}

// Next block time: the minimum over the new tend of the corrected particles
// (from correct_pass) and over every particle whose tend differs from the
// block time tb (this pass, taken before the correction so that its loads
// overlap the corrector's): a particle of the block read while some CTA
// corrects it shows either its old tend (== tb: skipped, its new value is in
// that CTA's minimum) or its new one (final).
__device__ long long scan_min_pass(const State &st, int64_t n, long long tb, int64_t g, int64_t G)
{
    const volatile long long *bits = reinterpret_cast<const volatile long long *>(st.tend);
    long long low = LLONG_MAX;
    for (int64_t i = g; i < n; i += G) {
        const long long v = bits[i];
        if (v != tb) low = min(low, v);
    }
    return low;
}

// One atomicMin per CTA of its threads' minima into sc->tnext_bits.
__device__ void publish_min(DevScalars *sc, long long low, long long *sh)
{
    low = block_min_ll(low, sh);
    if (threadIdx.x == 0 && low != LLONG_MAX) atomicMin((long long *)&sc->tnext_bits, low);
}

}  // namespace
}  // namespace hg
