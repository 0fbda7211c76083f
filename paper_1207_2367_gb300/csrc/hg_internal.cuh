// hg_internal.cuh -- data layout, launch plans and PTX helpers shared by the
// sm_103a kernels of the Hermite block-step engine.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "hg.h"

namespace hg {

// ---------------------------------------------------------------------------
// Device-side scalars of one context (one allocation).
// ---------------------------------------------------------------------------
struct DevScalars {
    double t_cur;          // current block time (written by the next-block pass)
    double t_stop;         // block steps whose time exceeds this are not taken
    int64_t m;             // size of the current block
    int64_t steps;         // block steps taken
    int64_t interactions;  // sum of m * n over those steps
    int32_t done;          // set when a next-block pass found t_next > t_stop
    int32_t err;           // error bits (ERR_*)
    int32_t flag;          // scratch result of validation kernels
    uint32_t slot;         // active-list entries taken so far by the fused selection
    int64_t plan[6];       // evaluation plan of the current block (a Plan, written on the device)
    int64_t tnext_bits;    // bit pattern of min_i tend_i (next-block pass 1, or the last correction)
    uint32_t arrive[4];    // CTAs done in next-block passes 1 and 2 and in the fused
                           // selection (the last one resets it); one spare
};

enum : int32_t { ERR_TIMEOUT = 1, ERR_BADIDX = 2, ERR_STATE = 4, ERR_VALUE = 8, ERR_BOUNDS = 16 };

// FP64 state of every particle at its own time, structure of arrays.
// tend = t + dt (exact: dyadic) is kept beside t and dt for the block selection.
// f32 (mixed contexts; nullptr otherwise): the FP32 roundings (d2f) of the
// fields the mixed predictor takes in FP32, four float4 per particle:
//   (v_x, v_y, v_z, m) (a_x, a_y, a_z, j_x) (j_y, j_z, s_x, s_y) (s_z, c_x, c_y, c_z)
// kept equal to d2f of the FP64 fields by every kernel that writes them, and
// rebuilt whenever the state is replaced from outside.
struct State {
    double *mass, *x, *v, *a, *j, *s, *c, *t, *dt, *tend;
    float4 *f32;
};
// Position of component k of each field in a particle's 16 FP32 values.
constexpr int kF32V = 0, kF32M = 3, kF32A = 4, kF32J = 7, kF32S = 10, kF32C = 13;

// ---------------------------------------------------------------------------
// Predicted j-records ("j-data"), npad entries (npad a multiple of the j-tile).
// Entries n..npad-1 are zero-mass padding far away from every particle, so
// tiles never need a bounds check.
//   mixed: records are interleaved in pairs (2P, 2P+1), so that one 16-byte
//          load gives the same two fields of both records as two register
//          pairs for the packed FP32 (f32x2) arithmetic.  Seven arrays of
//          npad / 2 entries, field f of record r at [r / 2].f[r % 2]:
//          p0 = (x_hi, y_hi)  p1 = (z_hi, m)  p2 = (x_lo, y_lo)  p3 = (z_lo, a_x)
//          p4 = (v_x, v_y)    p5 = (v_z, a_y)  (float4 each: f0 f0' f1 f1')
//          p6 = (a_z)         (float2: f0 f0')                   52 B/particle
//   fp64 : q0 = double2(x, y)  q1 = double2(z, m)  q2 = double2(v_x, v_y)
//          q3 = double2(v_z, a_x)  q4 = double2(a_y, a_z)          80 B/particle
// ---------------------------------------------------------------------------
struct Records {
    void *p[7];
};
constexpr int kMixedArrays = 7;

// One mixed j-record (FP32 fields) and its place in the pair-interleaved arrays.
struct MixedRecord {
    float xh, yh, zh, m, xl, yl, zl, ax, vx, vy, vz, ay, az;
};

constexpr int kEvalThreads = 128;
constexpr int kStages = 3;
constexpr int kTJMixed = 256;   // j-records per shared-memory tile, mixed
constexpr int kTJF64 = 128;     // j-records per shared-memory tile, fp64
constexpr int kIMixed = 1;      // i-particles held per thread, mixed
constexpr int kIF64 = 1;        // i-particles held per thread, fp64
constexpr int kMaxTPI = 64;
constexpr double kPadCoord = 1.0e18;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

// ---------------------------------------------------------------------------
// Work decomposition of one evaluation (Sect. 3 "Bfactor", redesigned): the m
// active particles form i-tiles of ti = (threads / tpi) * i_per_thread; each
// i-tile is split over b j-chunks of whole tiles ("j-split"), one work item
// per (i-tile, j-chunk).  tpi threads share an i-particle when m is small, so
// every lane has work; b spreads small blocks over all SMs.  A pure function
// of its arguments: the evaluation and the reduction compute the same plan.
// ---------------------------------------------------------------------------
struct Plan {
    int tpi, ti, b, variant;   // variant: which evaluation kernel runs the plan
    int64_t n_itiles, tiles_per_split, n_items;
};

constexpr int kTuneBuckets = HG_TUNE_BUCKETS;   // block sizes 2^k <= m < 2^(k+1)

// Inputs of the planner that do not change between block steps.  Variant 0
// holds i_per_thread particles per thread on `grid` persistent CTAs; variant 1
// (mixed, one system) holds ipt1 on grid1 CTAs.  One of its j-iterations costs
// weight1 / 100 of a variant-0 iteration when the plan needs several waves of
// work items (throughput-bound), weight1_one / 100 when one wave holds them all
// (latency-bound: a thread's longer iteration is not hidden by other warps).
struct PlanParams {
    int64_t ntiles;      // j-tiles of npad records
    int64_t pcap;        // b * m <= pcap (partial-sum capacity)
    int i_per_thread, tj, grid;
    int tpi_force, b_force;
    int c_tile, c_item;  // per-tile and per-item overhead, in j-iterations of one thread
    int variants;        // 1 or 2 evaluation kernels to choose from
    int ipt1, grid1, weight1, weight1_one;
    // Measured choices per block-size bucket (-1: cost model).  One system: a
    // candidate index; clusters: a batch code (see batch_knobs).
    int16_t tuned[kTuneBuckets];
};

__host__ __device__ inline int tune_bucket(int64_t m)
{
    int k = 0;
    while (k < kTuneBuckets - 1 && (m >> (k + 1)) > 0) ++k;
    return k;
}

// Block sizes at which the autotuner times every candidate plan of bucket k
// (2^k <= m < 2^(k+1)), the largest size tuned being mtop.  A stored plan serves
// the whole bucket and its wave count jumps with m, so one size is not enough:
// k = 0: 1; k = 1: 2, 3; k >= 2: 2^k * 5/4, 3/2, 7/4; each clamped to mtop,
// repeats dropped.  Returns how many (1 to 3).
__host__ __device__ inline int tune_point_add(int64_t v, int64_t mtop, int64_t (&pts)[3], int np)
{
    v = v < mtop ? v : mtop;
    if (np == 0 || pts[np - 1] != v) pts[np++] = v;
    return np;
}
__host__ __device__ inline int tune_points(int k, int64_t mtop, int64_t (&pts)[3])
{
    int np = 0;
    if (k == 0) {
        np = tune_point_add(1, mtop, pts, np);
    } else if (k == 1) {
        np = tune_point_add(2, mtop, pts, np);
        np = tune_point_add(3, mtop, pts, np);
    } else {
        for (int64_t f = 5; f <= 7; ++f) np = tune_point_add((f << k) / 4, mtop, pts, np);
    }
    return np;
}

// Candidate c in [0, variants * kPlanCandidates): variant c / kPlanCandidates,
// threads per i = 2^((c % kPlanCandidates) / 32), tiles per split plan_tps(c % 32).
constexpr int kPlanCandidates = 7 * 32;
constexpr int kPlanVariantsMax = 2;
__host__ __device__ inline int64_t plan_tps(int k)
{
    const int64_t t[32] = {1,  2,  3,  4,  5,  6,   7,   8,   9,   10,  11,   12,   13,   14,   15,   16,
                           20, 24, 32, 40, 48, 64, 96, 128, 192, 256, 384, 512, 1024, 2048, 4096, 8192};
    return t[k];
}

// ceil(a / b) for a >= 0, b > 0; 32-bit division when both fit (a 64-bit
// division is a long software sequence on the GPU and the device planner scores
// hundreds of candidates per block step).  Exact either way.
__host__ __device__ inline int64_t div_ceil(int64_t a, int64_t b)
{
    if (((uint64_t)a | (uint64_t)b) < 0x80000000ull) {
        const uint32_t a32 = (uint32_t)a, b32 = (uint32_t)b;
        return (int64_t)((a32 + b32 - 1u) / b32);
    }
    return (a + b - 1) / b;
}

// Fill p for candidate c and return its modelled cost (-1: not admissible).
// cost = waves * (tiles per item * (TJ / tpi + c_tile) + c_item), integers only
// so that host and device choose the same plan.
__host__ __device__ inline int64_t plan_candidate(int64_t m, const PlanParams &q, int c, Plan &p)
{
    const int v = c / kPlanCandidates;
    if (c < 0 || v >= q.variants) return -1;
    c -= v * kPlanCandidates;
    const int ipt = v ? q.ipt1 : q.i_per_thread, grid = v ? q.grid1 : q.grid;
    const int tpi = 1 << (c / 32);
    if (tpi > kMaxTPI || (q.tpi_force > 0 && tpi != q.tpi_force)) return -1;
    int64_t tps = plan_tps(c % 32);
    if (q.b_force > 0) {
        if (c % 32 != 0) return -1;
        const int64_t b = q.b_force < q.ntiles ? q.b_force : q.ntiles;
        tps = div_ceil(q.ntiles, b);
    }
    if (tps > q.ntiles) return -1;
    const int64_t b = div_ceil(q.ntiles, tps);
    const int64_t mm = m > 0 ? m : 1;
    if (b * mm > q.pcap && b > 1) return -1;
    p.tpi = tpi;
    p.ti = kEvalThreads / tpi * ipt;
    p.n_itiles = div_ceil(mm, p.ti);
    p.tiles_per_split = tps;
    p.b = (int)b;
    p.variant = v;
    p.n_items = p.n_itiles * b;
    const int64_t waves = div_ceil(p.n_items, grid);
    const int64_t w = v == 0 ? 100 : (waves > 1 ? q.weight1 : q.weight1_one);
    return waves * (tps * ((q.tj / tpi) * w + q.c_tile * 100) + q.c_item * 100);
}

__host__ __device__ inline int plan_total(const PlanParams &q) { return q.variants * kPlanCandidates; }

// The tuned candidate of m's bucket if there is one and it is admissible, else
// the cheapest admissible candidate of the cost model (ties: lowest index).
__host__ __device__ inline Plan make_plan(int64_t m, const PlanParams &q)
{
    Plan best{}, p{};
    const int tc = q.tuned[tune_bucket(m)];
    if (tc >= 0 && plan_candidate(m, q, tc, p) >= 0) return p;
    int64_t best_cost = -1;
    for (int c = 0; c < plan_total(q); ++c) {
        const int64_t cost = plan_candidate(m, q, c, p);
        if (cost >= 0 && (best_cost < 0 || cost < best_cost)) {
            best_cost = cost;
            best = p;
        }
    }
    if (best_cost < 0) plan_candidate(m, q, 0, best);   // unreachable: candidate 0 is admissible
    return best;
}

// Independent clusters in one context (nc == 0: a single system).  Particles of
// cluster c are [cl_off[c], cl_off[c+1]); its j-records occupy the 256-aligned
// range [rec_off[c], rec_off[c+1]) (zero-mass padding at the end), so every
// j-tile of a cluster starts on a tile boundary.  The per-step arrays form the
// work list written by the batch planning kernel.
struct BatchView {
    int32_t nc = 0;
    const int64_t *cl_off = nullptr;   // [nc+1] particle offsets
    const int64_t *rec_off = nullptr;  // [nc+1] record offsets (multiples of 256)
    const int32_t *rmap = nullptr;     // [n] record index of each particle
    const int32_t *cl_of = nullptr;    // [n] cluster of each particle
    int64_t *a_off = nullptr;          // [nc+1] first position of each cluster in the active list
    int64_t *item_off = nullptr;       // [nc+1] first work item of each cluster
    int64_t *part_off = nullptr;       // [nc+1] first partial-sum row of each cluster
    int64_t *pred_off = nullptr;       // [nc+1] prefix of the sizes of clusters with active particles
    int32_t *tpi_c = nullptr;          // [nc] threads per i-particle
    int32_t *b_c = nullptr;            // [nc] j-chunks
    int64_t *tps = nullptr;            // [1] tiles per j-chunk
};

constexpr int kBatchTpsMax = 64;   // tiles per j-chunk considered by the batch planner

// Knobs of the batch planner for a block of m: the j-split leaves at least
// 2^w_log work items per resident CTA; threads per i-particle are scaled by
// 2^tpi_shift.  Code w + 8 (s + 1); -1 (untuned): w = 1, s = 0.
struct BatchKnobs {
    int w_log, tpi_shift;
};
constexpr int kBatchWMax = 6;
__host__ __device__ inline bool batch_code_ok(int v)
{
    return v >= 0 && (v & 7) <= kBatchWMax && (v >> 3) <= 2;
}
__host__ __device__ inline BatchKnobs batch_knobs(int64_t m, const PlanParams &q)
{
    const int v = q.tuned[tune_bucket(m)];
    if (!batch_code_ok(v)) return BatchKnobs{1, 0};
    return BatchKnobs{v & 7, (v >> 3) - 1};
}

// Values per partial-sum row and per evaluated particle: acceleration, jerk and
// snap (3 each), then the noise scale sum_j m_j / (r_ij^2 + eps^2), an upper
// bound of sum_j |a_ij| (mixed kernels; the FP64 kernel writes 0).
constexpr int kOut = 10;

struct EvalArgs {
    Records rec{};
    int64_t npad = 0;
    int64_t n = 0;                     // particles (bounds of the active list's entries)
    int64_t pcap = 0;                  // rows of the partial-sum buffer
    const int32_t *idx = nullptr;      // active list (device)
    const int64_t *m_dev = nullptr;    // block size on the device (graph mode), or nullptr
    int64_t m_host = 0;                // block size when m_dev == nullptr
    const Plan *plan_dev = nullptr;    // plan on the device (graph mode), or nullptr
    Plan plan_host{};                  // plan when plan_dev == nullptr
    double *partial = nullptr;         // [b][m][kOut] partial sums
    double eps2 = 0.0;
    int guard = 0;                     // eps == 0: skip r^2 == 0 pairs
    uint32_t tx_extra = 0;             // testing: bytes expected per tile beyond those copied (0 normally)
    int32_t *err = nullptr;
    BatchView bv{};                    // clusters (bv.nc == 0: single system)
    // One system: a plan without j-split (b = 1) writes its sums straight into
    // ra/rj/rs [m][3] and the reduction kernel returns at once (direct_b1 = 1);
    // otherwise partials go to [b][m][kOut] and the reduction kernel sums them.
    int direct_b1 = 0;
    double *ra = nullptr, *rj = nullptr, *rs = nullptr;
    double *rn = nullptr;              // [m] noise scale (nullptr: not written)
};

// Planner inputs of one precision (hg_eval.cu): tiles, tile size, i per thread,
// overhead constants and the persistent grid of the evaluation kernel.
PlanParams plan_params(bool mixed, int64_t npad, int num_sms, int64_t pcap, int tpi_force, int b_force);

// Message of the last failed context-free call on this thread (hg_api.cu).
void set_call_error(const char *msg);

// Host-side launchers (hg_eval.cu).
cudaError_t eval_setup(int device);
int eval_grid(bool mixed, int num_sms);
// Evaluation of args: the precision's kernel on min(items, its grid) CTAs with
// a host plan, on its full persistent grid with a device plan (graph steps) or
// clusters.
cudaError_t launch_eval(bool mixed, const EvalArgs &args, int num_sms, cudaStream_t st);
// Kernels launch_eval issues for a device plan.
int eval_launches(bool mixed, const EvalArgs &args);
// Sums the b partials of each listed particle into res_{a,j,s} [m][3] and, when
// args.rn is set, the noise scale into args.rn [m] (grid-stride: grid CTAs of
// 256 threads, a few per SM).
cudaError_t launch_reduce(const EvalArgs &args, double *ra, double *rj, double *rs, int grid, cudaStream_t st);

// Bit patterns of IEEE-754 values (host and device).
__host__ __device__ __forceinline__ unsigned long long bits_of(double x)
{
#if defined(__CUDA_ARCH__)
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}
__host__ __device__ __forceinline__ unsigned int bits_of(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    unsigned int b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned int b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// FP64 <-> FP32 conversions done with integer operations on the IEEE-754
// encodings (binary64: 1 sign, 11 exponent bits, bias 1023, 52 fraction bits;
// binary32: 1, 8, bias 127, 23).  GB300's FP64 pipe, which also executes the
// hardware conversions, is the predictor's limit; the integer pipes are not.
// d2f: round to nearest, ties to even; results below the smallest normal float
// (2^-126) become zero of the same sign; magnitudes that round beyond the
// largest float become infinity of the same sign (IEEE overflow), infinities
// stay infinities and NaN stays NaN.
__host__ __device__ __forceinline__ float d2f(double x)
{
    const unsigned long long b = bits_of(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int be = (int)((b >> 52) & 0x7ffu);
    const int e = be - 1023 + 127;
    unsigned int m = (unsigned int)((b >> 29) & 0x7fffffu);
    const unsigned int rem = (unsigned int)b & 0x1fffffffu;
    m += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;   // may carry into e
    const unsigned int mag = ((unsigned int)e << 23) + m;                 // e = 254 carrying gives inf
    const bool nan = be == 0x7ff && (b & 0xfffffffffffffull) != 0ull;
    const unsigned int big = nan ? 0x7fc00000u : 0x7f800000u;             // overflow, inf or NaN
    return float_of(e <= 0 ? sign : (e >= 255 ? (sign | big) : (sign | mag)));
}

// Exact widening of a float that is zero, normal, infinite or NaN (subnormal
// floats, which the FP32 arithmetic here flushes, widen to zero).
__host__ __device__ __forceinline__ double f2d(float f)
{
    const unsigned int u = bits_of(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned int e = (u >> 23) & 0xffu;
    const unsigned long long frac = (unsigned long long)(u & 0x7fffffu) << 29;
    const unsigned long long mag = ((unsigned long long)(e + (1023u - 127u)) << 52) | frac;
    const unsigned long long special = (0x7ffull << 52) | frac;             // inf (frac 0) or NaN
    return double_of(e == 0u ? sign : (sign | (e == 255u ? special : mag)));
}

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and bulk (TMA) copies global -> shared.
// ---------------------------------------------------------------------------
#if defined(__CUDACC__)
// Bounds check of the checked build (compiled with -DHG_CHECKED): a false
// condition records ERR_BOUNDS in *err and the caller clamps or skips the
// access, so an out-of-range index becomes a reported error instead of a
// memory fault.  In the normal build the check compiles away (always true).
__device__ __forceinline__ bool in_bounds(bool ok, int32_t *err)
{
#if defined(HG_CHECKED)
    if (!ok) atomicOr(err, ERR_BOUNDS);
    return ok;
#else
    (void)ok;
    (void)err;
    return true;
#endif
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of bar, giving up after kWaitCycles (sets ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err)
{
    if (mbar_try_wait(bar, parity)) return true;
    long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > kWaitCycles) {
            atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// 1-D bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Hardware reciprocal square root (single MUFU instruction, flush-to-zero).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Mixed j-record r in the pair-interleaved arrays.
__device__ __forceinline__ void store_mixed_record(const Records &rec, int64_t r, const MixedRecord &v)
{
    const int64_t b = (r >> 1) * 4 + (r & 1);
    float *const *a = reinterpret_cast<float *const *>(rec.p);
    a[0][b] = v.xh; a[0][b + 2] = v.yh;
    a[1][b] = v.zh; a[1][b + 2] = v.m;
    a[2][b] = v.xl; a[2][b + 2] = v.yl;
    a[3][b] = v.zl; a[3][b + 2] = v.ax;
    a[4][b] = v.vx; a[4][b + 2] = v.vy;
    a[5][b] = v.vz; a[5][b + 2] = v.ay;
    a[6][(r >> 1) * 2 + (r & 1)] = v.az;
}

__device__ __forceinline__ MixedRecord load_mixed_record(const Records &rec, int64_t r)
{
    const int64_t b = (r >> 1) * 4 + (r & 1);
    const float *const *a = reinterpret_cast<const float *const *>(rec.p);
    MixedRecord v;
    v.xh = __ldcg(a[0] + b); v.yh = __ldcg(a[0] + b + 2);
    v.zh = __ldcg(a[1] + b); v.m = __ldcg(a[1] + b + 2);
    v.xl = __ldcg(a[2] + b); v.yl = __ldcg(a[2] + b + 2);
    v.zl = __ldcg(a[3] + b); v.ax = __ldcg(a[3] + b + 2);
    v.vx = __ldcg(a[4] + b); v.vy = __ldcg(a[4] + b + 2);
    v.vz = __ldcg(a[5] + b); v.ay = __ldcg(a[5] + b + 2);
    v.az = __ldcg(a[6] + (r >> 1) * 2 + (r & 1));
    return v;
}

// Packed FP32 pairs (PTX f32x2, sm_100 and later): two floats in one 64-bit
// register pair, each operation applied to both halves with FP32 rounding
// (round to nearest even), exactly as two scalar operations.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(f2_t r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
#endif

}  // namespace hg
