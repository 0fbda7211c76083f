// hg_eval.cu -- evaluation step (Sect. 3 item 2): acceleration, jerk and snap
// of the active i-particles against all predicted j-particles, on CUDA cores
// (the pair law is not a dense contraction), and the j-split reduction
// (Table 1, section 4).
//
// One persistent kernel per precision.  A CTA of 128 threads walks work items
// (i-tile, j-chunk).  j-records stream through a 3-stage ring of shared-memory
// tiles filled by 1-D bulk (TMA) copies completing on mbarriers; tpi threads
// share an i-particle and stride through each tile, then combine with warp
// shuffles (and shared memory for tpi > 32).  Partial sums of each j-chunk go
// to a [b][m][kOut] buffer that the reduction kernel sums in chunk order, so
// results do not depend on scheduling.  The mixed kernels also sum the noise
// scale sum_j m_j / (r_ij^2 + eps^2) >= sum_j |a_ij|: FP32 rounding of the pair
// terms leaves an error in a_i proportional to it, not to |a_i|, which can be
// hundreds of times smaller where the pull of the system cancels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr int kFold = 32;   // FP32 pair sums are folded into the compensated sum every kFold j's
// Smallest normal float.  With eps^2 below 2^-100 (the guarded evaluation) the
// softened r^2 of a particle with itself is zero or subnormal in FP32, where the
// flush-to-zero reciprocal square root gives infinity: such pairs are skipped.
constexpr float kFltMinNormal = 1.17549435e-38f;

// ------------------------------------------------------------------------
// Mixed precision: FP32 pair arithmetic, double-single position differences,
// Kahan-compensated FP32 sums (Sect. 5.7 hybrid precision, redesigned).
// ------------------------------------------------------------------------
// Each lane takes the j-records two at a time (one pair of the interleaved
// layout) and evaluates both pairs (i, 2P) and (i, 2P+1) with packed f32x2
// operations: the halves of every register pair belong to the two j, the
// i-particle's values are duplicated into both halves once per work item.
// One packed instruction does the FP32 work of two, so the issue slots per
// pair interaction halve and the FP32 pipe (not instruction issue) becomes
// the limit.  One i-particle per thread, 3 CTAs per SM: measured against two
// per thread (2 CTAs per SM), two j-pairs per iteration, and 4 CTAs per SM,
// it was faster overall and within 1 % where another form won.
template <int IPT>
struct Mixed {
    static constexpr int TJ = kTJMixed;
    static constexpr int TP = TJ / 2;   // record pairs per tile
    static constexpr int I = IPT;
    static constexpr int kMinBlocks = 3;
    static constexpr int kVariant = 0;
    static constexpr uint32_t kStageBytes = TJ * 52;
    struct IData {
        f2_t xh, yh, zh, xl, yl, zl, vx, vy, vz, ax, ay, az;   // (v, v) duplicated
    };
    struct ITile {
        IData d[I];
        int rid[I];   // record index of each i-particle (its own pair is left out of the noise scale)
    };
    struct Acc {
        float hi[I][9], lo[I][9];
        float n[I];   // noise scale (positive terms, plain sums of kFold-term chunks)
    };
    typedef float Eps;

    __device__ static void load_i(const Records &rec, int r, IData &d)
    {
        const MixedRecord v = load_mixed_record(rec, r);
        d.xh = f2_pack(v.xh, v.xh); d.yh = f2_pack(v.yh, v.yh); d.zh = f2_pack(v.zh, v.zh);
        d.xl = f2_pack(v.xl, v.xl); d.yl = f2_pack(v.yl, v.yl); d.zl = f2_pack(v.zl, v.zl);
        d.vx = f2_pack(v.vx, v.vx); d.vy = f2_pack(v.vy, v.vy); d.vz = f2_pack(v.vz, v.vz);
        d.ax = f2_pack(v.ax, v.ax); d.ay = f2_pack(v.ay, v.ay); d.az = f2_pack(v.az, v.az);
    }

    __device__ static void zero(Acc &a)
    {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            a.n[k] = 0.f;
#pragma unroll
            for (int c = 0; c < 9; ++c) a.hi[k][c] = a.lo[k][c] = 0.f;
        }
    }

    __device__ static void load(const Records &rec, const int (&ids)[I], ITile &t)
    {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            load_i(rec, ids[k], t.d[k]);
            t.rid[k] = ids[k];
        }
    }

    __device__ static void issue(const Records &rec, int64_t tile, unsigned char *dst, uint64_t *bar,
                                 uint32_t tx_extra)
    {
        const int64_t p0 = tile * TP;
        mbar_arrive_expect_tx(bar, kStageBytes + tx_extra);
#pragma unroll
        for (int q = 0; q < 6; ++q)
            bulk_g2s(dst + q * TP * 16, static_cast<const float4 *>(rec.p[q]) + p0, TP * 16, bar);
        bulk_g2s(dst + 6 * TP * 16, static_cast<const float2 *>(rec.p[6]) + p0, TP * 8, bar);
    }

    // Pairs (i, 2P) and (i, 2P+1): r_ij = r_j - r_i from (hi, lo) parts, v_ij,
    // a_ij, softened r^2, alpha r^2 = r.v, beta r^2 = v^2 + r.a + alpha^2 r^2, and
    // A = m r / r^3, J = m v / r^3 - 3 alpha A, S = m a / r^3 - 6 alpha J - 3 beta A,
    // written as A = q r, J = q w, S = q u with q = m / r^3, w = v - 3 alpha r and
    // u = a - 6 alpha w - 3 beta r, so that each sum takes one FMA per component.
    // ns gathers m / (r^2 + eps^2) (>= |A|) times keep: (1, 1), or 0 in the half
    // holding the i-particle itself.
    template <bool GUARD>
    __device__ __forceinline__ static void pair(const IData &d, const float4 q0, const float4 q1,
                                                const float4 q2, const float4 q3, const float4 q4,
                                                const float4 q5, const float2 q6, const f2_t eps2, f2_t keep,
                                                f2_t (&s)[9], f2_t &ns)
    {
        const f2_t k_m3 = f2_pack(-3.f, -3.f);
        const f2_t dx = f2_add(f2_sub(f2_pack(q0.x, q0.y), d.xh), f2_sub(f2_pack(q2.x, q2.y), d.xl));
        const f2_t dy = f2_add(f2_sub(f2_pack(q0.z, q0.w), d.yh), f2_sub(f2_pack(q2.z, q2.w), d.yl));
        const f2_t dz = f2_add(f2_sub(f2_pack(q1.x, q1.y), d.zh), f2_sub(f2_pack(q3.x, q3.y), d.zl));
        const f2_t dvx = f2_sub(f2_pack(q4.x, q4.y), d.vx);
        const f2_t dvy = f2_sub(f2_pack(q4.z, q4.w), d.vy);
        const f2_t dvz = f2_sub(f2_pack(q5.x, q5.y), d.vz);
        const f2_t dax = f2_sub(f2_pack(q3.z, q3.w), d.ax);
        const f2_t day = f2_sub(f2_pack(q5.z, q5.w), d.ay);
        const f2_t daz = f2_sub(f2_pack(q6.x, q6.y), d.az);
        const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_fma(dx, dx, eps2)));
        const float2 r2s = f2_unpack(r2);
        float y0 = rsqrt_approx(r2s.x), y1 = rsqrt_approx(r2s.y);
        if (GUARD) {   // r^2 below FP32's normal range: a pair at zero distance, skipped
            y0 = r2s.x >= kFltMinNormal ? y0 : 0.f;
            y1 = r2s.y >= kFltMinNormal ? y1 : 0.f;
        }
        // The hardware reciprocal square root is used as it is: a Newton-Raphson
        // step in FP32 cannot improve on its ~1-ulp result, and measured against
        // the FP64 kernel it changed the normwise acc / jerk / snap errors by < 10 %
        // (3.3e-8 / 2.2e-7 / 3.8e-7 at N = 131072) while costing 4 of the pair's 59
        // packed operations (4.5-4.9 % of the evaluation's time).
        const f2_t y = f2_pack(y0, y1);
        const f2_t rinv2 = f2_mul(y, y);
        const f2_t mr2 = f2_mul(f2_pack(q1.z, q1.w), rinv2);
        const f2_t q = f2_mul(mr2, y);
        ns = f2_fma(mr2, keep, ns);
        const f2_t rv = f2_fma(dz, dvz, f2_fma(dy, dvy, f2_mul(dx, dvx)));
        const f2_t v2ra =
            f2_fma(dz, daz, f2_fma(dy, day, f2_fma(dx, dax, f2_fma(dvz, dvz, f2_fma(dvy, dvy, f2_mul(dvx, dvx))))));
        const f2_t alpha = f2_mul(rv, rinv2);
        const f2_t beta = f2_fma(alpha, alpha, f2_mul(v2ra, rinv2));
        const f2_t a3 = f2_mul(k_m3, alpha);
        const f2_t a6 = f2_add(a3, a3), b3 = f2_mul(k_m3, beta);
        const f2_t wx = f2_fma(a3, dx, dvx), wy = f2_fma(a3, dy, dvy), wz = f2_fma(a3, dz, dvz);
        s[0] = f2_fma(q, dx, s[0]);
        s[1] = f2_fma(q, dy, s[1]);
        s[2] = f2_fma(q, dz, s[2]);
        s[3] = f2_fma(q, wx, s[3]);
        s[4] = f2_fma(q, wy, s[4]);
        s[5] = f2_fma(q, wz, s[5]);
        s[6] = f2_fma(q, f2_fma(b3, dx, f2_fma(a6, wx, dax)), s[6]);
        s[7] = f2_fma(q, f2_fma(b3, dy, f2_fma(a6, wy, day)), s[7]);
        s[8] = f2_fma(q, f2_fma(b3, dz, f2_fma(a6, wz, daz)), s[8]);
    }

    // Kahan step: hi + x with the running compensation lo (true sum = hi - lo).
    __device__ __forceinline__ static void kahan(float &hi, float &lo, float x)
    {
        const float y = x - lo;
        const float t = hi + y;
        lo = (t - hi) - y;
        hi = t;
    }

    // Pair (i, record pair jp) of every i-particle of the lane.
    template <bool GUARD, bool MASK>
    __device__ __forceinline__ static void pair_step(const float4 *a0, const float2 *a6, int jp, const ITile &iv,
                                                     f2_t eps2, const int (&selfp)[I], const f2_t (&selfk)[I],
                                                     f2_t (&ch)[I][9], f2_t (&cn)[I])
    {
        const f2_t one2 = f2_pack(1.f, 1.f);
        const float4 q0 = a0[jp], q1 = a0[TP + jp], q2 = a0[2 * TP + jp], q3 = a0[3 * TP + jp],
                     q4 = a0[4 * TP + jp], q5 = a0[5 * TP + jp];
        const float2 q6 = a6[jp];
#pragma unroll
        for (int k = 0; k < I; ++k)
            pair<GUARD>(iv.d[k], q0, q1, q2, q3, q4, q5, q6, eps2, (MASK && jp == selfp[k]) ? selfk[k] : one2,
                        ch[k], cn[k]);
    }

    // The pairs of one tile: TP / tpi record pairs per lane, folded into the
    // compensated sums every kFold / 2.  MASK: some lane's own record is in the
    // tile (pair selfp[k], keep-mask selfk[k]); without it the noise scale needs
    // no mask.  TPI > 0: tpi known at compile time, so that the pairs of a fold
    // are unrolled with constant shared-memory offsets (measured: 9 % faster than
    // the loop with a run-time stride at tpi = 1); TPI = 0: any tpi.
    template <bool GUARD, bool MASK, int TPI>
    __device__ __forceinline__ static void tile_pairs(const float4 *a0, const float2 *a6, int tpi_rt, int lane_j,
                                                      const ITile &iv, Acc &acc, f2_t eps2, const int (&selfp)[I],
                                                      const f2_t (&selfk)[I])
    {
        constexpr int kF = kFold / 2;
        if constexpr (TPI > 0) {
            constexpr int kPpt = TP / TPI;                    // pairs per lane in this tile
            constexpr int kU = kPpt < kF ? kPpt : kF;         // pairs per fold
            const int lj = TPI == 1 ? 0 : lane_j;
            for (int g = 0; g < kPpt; g += kU) {
                f2_t ch[I][9], cn[I];
                zero_chunk(ch, cn);
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    pair_step<GUARD, MASK>(a0, a6, (g + u) * TPI + lj, iv, eps2, selfp, selfk, ch, cn);
                fold_chunk(acc, ch, cn);
            }
        } else {
            const int ppt = TP >> (__ffs(tpi_rt) - 1);        // tpi a power of two
            const int fold = ppt < kF ? ppt : kF;
            for (int g = 0; g < ppt; g += fold) {
                f2_t ch[I][9], cn[I];
                zero_chunk(ch, cn);
                for (int u = 0; u < fold; ++u)
                    pair_step<GUARD, MASK>(a0, a6, (g + u) * tpi_rt + lane_j, iv, eps2, selfp, selfk, ch, cn);
                fold_chunk(acc, ch, cn);
            }
        }
    }

    __device__ __forceinline__ static void zero_chunk(f2_t (&ch)[I][9], f2_t (&cn)[I])
    {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            cn[k] = 0ull;
#pragma unroll
            for (int c = 0; c < 9; ++c) ch[k][c] = 0ull;
        }
    }

    // The FP32 chunk sums of a fold into the compensated sums.
    __device__ __forceinline__ static void fold_chunk(Acc &acc, const f2_t (&ch)[I][9], const f2_t (&cn)[I])
    {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const float2 nn = f2_unpack(cn[k]);
            acc.n[k] += nn.x + nn.y;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                const float2 v = f2_unpack(ch[k][c]);
                kahan(acc.hi[k][c], acc.lo[k][c], v.x + v.y);
            }
        }
    }

    // Compile-time strides for 1, 2 and 4 threads per particle (the plans of large
    // blocks); copies for every tpi up to 64 measured slower everywhere (more code).
    template <bool GUARD, bool MASK>
    __device__ __forceinline__ static void tile_by_tpi(const float4 *a0, const float2 *a6, int tpi, int lane_j,
                                                       const ITile &iv, Acc &acc, f2_t eps2, const int (&selfp)[I],
                                                       const f2_t (&selfk)[I])
    {
        if (tpi == 1)
            tile_pairs<GUARD, MASK, 1>(a0, a6, tpi, lane_j, iv, acc, eps2, selfp, selfk);
        else if (tpi == 2)
            tile_pairs<GUARD, MASK, 2>(a0, a6, tpi, lane_j, iv, acc, eps2, selfp, selfk);
        else if (tpi == 4)
            tile_pairs<GUARD, MASK, 4>(a0, a6, tpi, lane_j, iv, acc, eps2, selfp, selfk);
        else
            tile_pairs<GUARD, MASK, 0>(a0, a6, tpi, lane_j, iv, acc, eps2, selfp, selfk);
    }

    // tile: absolute index of the j-tile, to find the pair holding each
    // i-particle's own record.  Only the tile holding a lane's own record runs
    // the masked loop (warp-uniform choice): the mask's compare and selects in
    // every pair iteration of the others cost 3.5 % of the evaluation's time.
    template <bool GUARD>
    __device__ static void tile(const unsigned char *sb, int tpi, int lane_j, const ITile &iv, Acc &acc,
                                Eps eps2s, int64_t tile)
    {
        const float4 *a0 = reinterpret_cast<const float4 *>(sb);
        const float2 *a6 = reinterpret_cast<const float2 *>(a0 + 6 * TP);
        const f2_t eps2 = f2_pack(eps2s, eps2s);
        int selfp[I];   // pair of this tile holding i-particle k's own record, or -1
        f2_t selfk[I];  // keep-mask of that pair
        bool mine = false;
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int64_t r = iv.rid[k];
            selfp[k] = (r / TJ == tile) ? (int)((r % TJ) >> 1) : -1;
            selfk[k] = (r & 1) ? f2_pack(1.f, 0.f) : f2_pack(0.f, 1.f);
            mine = mine || selfp[k] >= 0;
        }
        if (__any_sync(0xffffffffu, mine))
            tile_by_tpi<GUARD, true>(a0, a6, tpi, lane_j, iv, acc, eps2, selfp, selfk);
        else
            tile_by_tpi<GUARD, false>(a0, a6, tpi, lane_j, iv, acc, eps2, selfp, selfk);
    }

    // Compensated pairs (true value hi - lo) added without rounding loss in hi:
    // two-sum s + e = hi1 + hi2 exactly (Knuth), then lo = lo1 + lo2 - e.
    __device__ __forceinline__ static void add_pair(float &hi, float &lo, float hi2, float lo2)
    {
        const float s = hi + hi2;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (hi2 - bb);
        hi = s;
        lo = (lo + lo2) - e;
    }

    // Sum the tpi lanes sharing an i-particle (fixed xor tree; shared memory
    // across warps for tpi = 64) in FP32 pairs, then widen once: the leader lanes
    // (lane_j == 0) hold out = hi - lo in FP64.  On GB300 an FP64 warp
    // instruction costs ~64 cycles, so the tree stays in FP32 and the widening
    // uses the integer f2d.
    __device__ static void epilogue(Acc &a, int tpi, int tid, double *red, double (&out)[I][kOut])
    {
        const int wspan = tpi < 32 ? tpi : 32;
        for (int off = 1; off < wspan; off <<= 1) {
#pragma unroll
            for (int k = 0; k < I; ++k) {
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    const float h2 = __shfl_xor_sync(0xffffffffu, a.hi[k][c], off);
                    const float l2 = __shfl_xor_sync(0xffffffffu, a.lo[k][c], off);
                    add_pair(a.hi[k][c], a.lo[k][c], h2, l2);
                }
                a.n[k] += __shfl_xor_sync(0xffffffffu, a.n[k], off);
            }
        }
        if (tpi > 32) {
            float2 *r2 = reinterpret_cast<float2 *>(red);
            const int warp = tid >> 5, lane = tid & 31, wpg = tpi >> 5;
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < I; ++k) {
#pragma unroll
                    for (int c = 0; c < 9; ++c)
                        r2[(warp * I + k) * kOut + c] = make_float2(a.hi[k][c], a.lo[k][c]);
                    r2[(warp * I + k) * kOut + 9] = make_float2(a.n[k], 0.f);
                }
            }
            __syncthreads();
            if (lane == 0 && (warp % wpg) == 0) {
#pragma unroll
                for (int k = 0; k < I; ++k) {
#pragma unroll
                    for (int c = 0; c < 9; ++c)
                        for (int g = 1; g < wpg; ++g) {
                            const float2 v = r2[((warp + g) * I + k) * kOut + c];
                            add_pair(a.hi[k][c], a.lo[k][c], v.x, v.y);
                        }
                    for (int g = 1; g < wpg; ++g) a.n[k] += r2[((warp + g) * I + k) * kOut + 9].x;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < I; ++k) {
#pragma unroll
            for (int c = 0; c < 9; ++c) out[k][c] = f2d(a.hi[k][c]) - f2d(a.lo[k][c]);
            out[k][9] = f2d(a.n[k]);
        }
    }
};

// ------------------------------------------------------------------------
// FP64 throughout.
// ------------------------------------------------------------------------
struct F64 {
    static constexpr int TJ = kTJF64;
    static constexpr int I = kIF64;
    static constexpr int kMinBlocks = 2;
    static constexpr int kVariant = 0;
    static constexpr uint32_t kStageBytes = TJ * 80;
    struct IData {
        double x, y, z, vx, vy, vz, ax, ay, az;
    };
    struct ITile {
        IData d[I];
    };
    struct Acc {
        double s[I][9];
    };
    typedef double Eps;

    __device__ static void load_i(const Records &rec, int i, IData &d)
    {
        const double2 q0 = __ldcg(static_cast<const double2 *>(rec.p[0]) + i);
        const double2 q1 = __ldcg(static_cast<const double2 *>(rec.p[1]) + i);
        const double2 q2 = __ldcg(static_cast<const double2 *>(rec.p[2]) + i);
        const double2 q3 = __ldcg(static_cast<const double2 *>(rec.p[3]) + i);
        const double2 q4 = __ldcg(static_cast<const double2 *>(rec.p[4]) + i);
        d.x = q0.x; d.y = q0.y; d.z = q1.x;
        d.vx = q2.x; d.vy = q2.y; d.vz = q3.x;
        d.ax = q3.y; d.ay = q4.x; d.az = q4.y;
    }

    __device__ static void zero(Acc &a)
    {
#pragma unroll
        for (int k = 0; k < I; ++k)
#pragma unroll
            for (int c = 0; c < 9; ++c) a.s[k][c] = 0.0;
    }

    __device__ static void load(const Records &rec, const int (&ids)[I], ITile &t)
    {
#pragma unroll
        for (int k = 0; k < I; ++k) load_i(rec, ids[k], t.d[k]);
    }

    __device__ static void issue(const Records &rec, int64_t tile, unsigned char *dst, uint64_t *bar,
                                 uint32_t tx_extra)
    {
        const int64_t j0 = tile * TJ;
        mbar_arrive_expect_tx(bar, kStageBytes + tx_extra);
#pragma unroll
        for (int q = 0; q < 5; ++q)
            bulk_g2s(dst + q * TJ * 16, static_cast<const double2 *>(rec.p[q]) + j0, TJ * 16, bar);
    }

    template <bool GUARD>
    __device__ __forceinline__ static void pair(const IData &d, const double2 q0, const double2 q1,
                                                const double2 q2, const double2 q3, const double2 q4,
                                                const double eps2, double (&s)[9])
    {
        const double dx = q0.x - d.x, dy = q0.y - d.y, dz = q1.x - d.z;
        const double dvx = q2.x - d.vx, dvy = q2.y - d.vy, dvz = q3.x - d.vz;
        const double dax = q3.y - d.ax, day = q4.x - d.ay, daz = q4.y - d.az;
        const double r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
        double rinv = rsqrt(r2);
        if (GUARD) rinv = (r2 > 0.0) ? rinv : 0.0;
        const double rinv2 = rinv * rinv;
        const double q = q1.y * rinv * rinv2;
        const double rv = fma(dz, dvz, fma(dy, dvy, dx * dvx));
        const double v2ra = fma(dz, daz, fma(dy, day, fma(dx, dax, fma(dvz, dvz, fma(dvy, dvy, dvx * dvx)))));
        const double alpha = rv * rinv2;
        const double beta = fma(alpha, alpha, v2ra * rinv2);
        const double a3 = -3.0 * alpha;
        const double a6 = a3 + a3, b3 = -3.0 * beta;
        const double wx = fma(a3, dx, dvx), wy = fma(a3, dy, dvy), wz = fma(a3, dz, dvz);
        s[0] = fma(q, dx, s[0]);
        s[1] = fma(q, dy, s[1]);
        s[2] = fma(q, dz, s[2]);
        s[3] = fma(q, wx, s[3]);
        s[4] = fma(q, wy, s[4]);
        s[5] = fma(q, wz, s[5]);
        s[6] = fma(q, fma(b3, dx, fma(a6, wx, dax)), s[6]);
        s[7] = fma(q, fma(b3, dy, fma(a6, wy, day)), s[7]);
        s[8] = fma(q, fma(b3, dz, fma(a6, wz, daz)), s[8]);
    }

    template <bool GUARD>
    __device__ static void tile(const unsigned char *sb, int tpi, int lane_j, const ITile &iv, Acc &acc,
                                Eps eps2, int64_t)
    {
        const double2 *q0 = reinterpret_cast<const double2 *>(sb);
        const int jpt = TJ >> (__ffs(tpi) - 1);   // tpi a power of two
#pragma unroll 2
        for (int u = 0; u < jpt; ++u) {
            const int jj = u * tpi + lane_j;
            const double2 a = q0[jj], b = q0[TJ + jj], c = q0[2 * TJ + jj], d = q0[3 * TJ + jj],
                          e = q0[4 * TJ + jj];
#pragma unroll
            for (int k = 0; k < I; ++k) pair<GUARD>(iv.d[k], a, b, c, d, e, eps2, acc.s[k]);
        }
    }

    // Sum the tpi lanes sharing an i-particle (fixed xor tree; shared memory
    // across warps for tpi = 64): the leader lanes (lane_j == 0) hold out.  No
    // noise scale (out[k][9] = 0): the FP64 path needs no noise floor.
    __device__ static void epilogue(Acc &a, int tpi, int tid, double *red, double (&out)[I][kOut])
    {
#pragma unroll
        for (int k = 0; k < I; ++k) {
#pragma unroll
            for (int c = 0; c < 9; ++c) out[k][c] = a.s[k][c];
            out[k][9] = 0.0;
        }
        const int wspan = tpi < 32 ? tpi : 32;
        for (int off = 1; off < wspan; off <<= 1) {
#pragma unroll
            for (int k = 0; k < I; ++k)
#pragma unroll
                for (int c = 0; c < 9; ++c) out[k][c] += __shfl_xor_sync(0xffffffffu, out[k][c], off);
        }
        if (tpi > 32) {
            const int warp = tid >> 5, lane = tid & 31, wpg = tpi >> 5;
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < I; ++k)
#pragma unroll
                    for (int c = 0; c < 9; ++c) red[(warp * I + k) * kOut + c] = out[k][c];
            }
            __syncthreads();
            if (lane == 0 && (warp % wpg) == 0) {
#pragma unroll
                for (int k = 0; k < I; ++k)
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        double s = red[(warp * I + k) * kOut + c];
                        for (int g = 1; g < wpg; ++g) s += red[((warp + g) * I + k) * kOut + c];
                        out[k][c] = s;
                    }
            }
            __syncthreads();
        }
    }
};

typedef Mixed<kIMixed> MixedEval;

template <class P>
constexpr size_t smem_bytes()
{
    return (size_t)kStages * P::kStageBytes + kStages * sizeof(uint64_t) +
           (kEvalThreads / 32) * P::I * kOut * sizeof(double);
}

// The work items (i-tile, j-chunk) of one evaluation that this CTA takes
// (items blockIdx.x, blockIdx.x + gridDim.x, ...): the body of k_eval.  bars: the kStages
// initialised mbarriers of the tile ring; seq: tiles this CTA consumed so far
// (their phase bookkeeping, carried across calls).  False when a bounded wait
// expired (ERR_TIMEOUT is set; the copies in flight have been waited for).
template <class P, bool GUARD>
__device__ bool eval_items(const EvalArgs &args, int64_t m, const Plan &pl, unsigned char *smem, uint64_t *bars,
                           double *red, uint32_t &seq)
{
    const int tid = threadIdx.x;
    const BatchView &bv = args.bv;
    const bool batch = bv.nc > 0;
    if (!batch && pl.variant != P::kVariant) return true;   // a plan for another kernel (none at present)
    const int64_t n_items = batch ? bv.item_off[bv.nc] : pl.n_items;
    const int64_t tps = batch ? *bv.tps : pl.tiles_per_split;
    const typename P::Eps eps2 = (typename P::Eps)args.eps2;

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        // Decode the item: active positions [q_begin, q_end) of this i-tile's
        // system, first i-position of the tile, j-tiles [tbase, tbase + nt),
        // and the partial-sum row of position q (rbase + q).
        int tpi;
        int64_t q_tile, q_end, tbase, rbase, nt64;
        if (batch) {
            int lo = 0, hi = bv.nc - 1;            // last cluster with item_off[c] <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bv.item_off[mid] <= item) lo = mid; else hi = mid - 1;
            }
            const int c = lo;
            tpi = bv.tpi_c[c];
            const int64_t b = bv.b_c[c];
            const int64_t local = item - bv.item_off[c];
            const int64_t itile = local / b, split = local - itile * b;
            const int64_t qb = bv.a_off[c], mc = bv.a_off[c + 1] - qb;
            const int64_t ti = kEvalThreads / tpi * P::I;
            q_tile = qb + itile * ti;
            q_end = qb + mc;
            const int64_t t0 = bv.rec_off[c] / P::TJ, ntc = (bv.rec_off[c + 1] - bv.rec_off[c]) / P::TJ;
            tbase = t0 + split * tps;
            nt64 = ntc - split * tps < tps ? ntc - split * tps : tps;
            rbase = bv.part_off[c] + split * mc - qb;
        } else {
            tpi = pl.tpi;
            const int64_t itile = item / pl.b, split = item - itile * pl.b;
            const int64_t ntiles = args.npad / P::TJ;
            q_tile = itile * pl.ti;
            q_end = m;
            tbase = split * tps;
            nt64 = ntiles - tbase < tps ? ntiles - tbase : tps;
            rbase = split * m;
        }
        if (!in_bounds(tbase >= 0 && nt64 >= 0 && tbase + nt64 <= args.npad / P::TJ, args.err)) nt64 = 0;
        const int nt = (int)nt64;
        const int lane_j = tid & (tpi - 1);
        const int slot = tid >> (__ffs(tpi) - 1);   // tid / tpi (a power of two)

        typename P::ITile iv;
        int64_t qi[P::I];
        int ids[P::I];
#pragma unroll
        for (int k = 0; k < P::I; ++k) {
            qi[k] = q_tile + (int64_t)slot * P::I + k;
            int64_t qc = qi[k] < q_end ? qi[k] : q_end - 1;
            if (!in_bounds(qc >= 0 && qc < args.n, args.err)) qc = 0;
            int32_t i = __ldcg(args.idx + qc);
            if (!in_bounds(i >= 0 && (int64_t)i < args.n, args.err)) i = 0;
            int32_t r = batch ? bv.rmap[i] : i;
            if (!in_bounds(r >= 0 && (int64_t)r < args.npad, args.err)) r = 0;
            ids[k] = r;
        }
        P::load(args.rec, ids, iv);
        typename P::Acc acc;
        P::zero(acc);

        if (tid == 0) {
            const int pre = nt < kStages ? nt : kStages;
            for (int s = 0; s < pre; ++s) {
                const int st = (int)((seq + s) % kStages);
                P::issue(args.rec, tbase + s, smem + st * P::kStageBytes, &bars[st], args.tx_extra);
            }
        }
        for (int t = 0; t < nt; ++t) {
            const uint32_t sq = seq + (uint32_t)t;
            const int st = (int)(sq % kStages);
            const bool ok = mbar_wait_bounded(&bars[st], (sq / kStages) & 1u, args.err);
            if (ok) P::template tile<GUARD>(smem + st * P::kStageBytes, tpi, lane_j, iv, acc, eps2, tbase + t);
            if (__syncthreads_or(!ok)) {
                // A copy never completed: wait (bounded) for what is still in flight, then leave.
                if (tid == 0) {
                    const int issued = (t + kStages) < nt ? (t + kStages) : nt;
                    for (int u = t; u < issued; ++u) {
                        const uint32_t q = seq + (uint32_t)u;
                        mbar_wait_bounded(&bars[q % kStages], (q / kStages) & 1u, args.err);
                    }
                }
                return false;
            }
            if (tid == 0 && t + kStages < nt) {
                fence_proxy_async();
                P::issue(args.rec, tbase + t + kStages, smem + st * P::kStageBytes, &bars[st], args.tx_extra);
            }
        }
        seq += (uint32_t)nt;

        double out[P::I][kOut];
        P::epilogue(acc, tpi, tid, red, out);
        if (!batch && args.direct_b1 && pl.b == 1) {   // no j-split: these are the results
            if (lane_j == 0) {
#pragma unroll
                for (int k = 0; k < P::I; ++k)
                    if (qi[k] < q_end) {
#pragma unroll
                        for (int c = 0; c < 9; ++c) {
                            double *dst = c < 3 ? args.ra : (c < 6 ? args.rj : args.rs);
                            dst[qi[k] * 3 + c % 3] = out[k][c];
                        }
                        if (args.rn) args.rn[qi[k]] = out[k][9];
                    }
            }
            continue;
        }
        if (lane_j == 0) {
#pragma unroll
            for (int k = 0; k < P::I; ++k) {
                if (qi[k] < q_end && in_bounds(rbase + qi[k] >= 0 && rbase + qi[k] < args.pcap, args.err)) {
                    double *dst = args.partial + (rbase + qi[k]) * kOut;
#pragma unroll
                    for (int c = 0; c < kOut; ++c) dst[c] = out[k][c];
                }
            }
        }
    }
    return true;
}

template <class P, bool GUARD>
__global__ void __launch_bounds__(kEvalThreads, P::kMinBlocks) k_eval(const EvalArgs args)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * P::kStageBytes);
    double *red = reinterpret_cast<double *>(bars + kStages);
    const int64_t m = args.m_dev ? *args.m_dev : args.m_host;
    if (m <= 0) return;
    const Plan pl = args.plan_dev ? *args.plan_dev : args.plan_host;
    const int64_t n_items = args.bv.nc > 0 ? args.bv.item_off[args.bv.nc] : pl.n_items;
    if ((int64_t)blockIdx.x >= n_items) return;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t seq = 0;   // tiles consumed so far by this CTA (mbarrier phase bookkeeping)
    eval_items<P, GUARD>(args, m, pl, smem, bars, red, seq);
}

// Table 1 section 4: sum the b j-chunk partials of every listed particle in
// chunk order and scatter them to acc/jerk/snap [m][3] (and the noise scale to
// args.rn [m] when it is set).
__device__ __forceinline__ void put_result(const EvalArgs &a, double *ra, double *rj, double *rs, int64_t q, int c,
                                           double v)
{
    if (c == 9) {
        if (a.rn) a.rn[q] = v;
        return;
    }
    double *dst = c < 3 ? ra : (c < 6 ? rj : rs);
    dst[q * 3 + (c % 3)] = v;
}

// The reduction's values taken by global thread g of G threads (grid-stride):
// the body of k_reduce.
// Each (particle, value) sum has a fixed order whichever thread takes it.
__device__ void reduce_values(const EvalArgs &args, int64_t m, const Plan &pl, double *ra, double *rj, double *rs,
                              int64_t g, int64_t G)
{
    if (args.bv.nc == 0 && args.direct_b1 && pl.b == 1) return;   // the evaluation wrote the results
    const int64_t total = m * kOut;
    if (args.bv.nc > 0) {
        // Clusters: the chunks of position q are rows part_off[c] + s * m_c + (q - a_off[c]).
        const BatchView &bv = args.bv;
        for (int64_t e = g; e < total; e += G) {
            const int64_t q = e / kOut;
            const int cv = (int)(e - q * kOut);
            const int32_t iq = __ldcg(args.idx + q);
            if (!in_bounds(iq >= 0 && (int64_t)iq < args.n, args.err)) continue;
            const int c = bv.cl_of[iq];
            const int64_t qb = bv.a_off[c], mc = bv.a_off[c + 1] - qb;
            const int64_t row0 = bv.part_off[c] + (q - qb);
            const int b = bv.b_c[c];
            if (!in_bounds(row0 >= 0 && row0 + (int64_t)(b - 1) * mc < args.pcap, args.err)) continue;
            double s = 0.0;
            for (int sp = 0; sp < b; ++sp) s += __ldcg(args.partial + (row0 + (int64_t)sp * mc) * kOut + cv);
            put_result(args, ra, rj, rs, q, cv, s);
        }
        return;
    }
    if (!in_bounds((int64_t)pl.b * m <= args.pcap, args.err)) return;
    if (pl.b <= 32) {
        // Few chunks: one thread per (particle, value), chunks in order.
        for (int64_t e = g; e < total; e += G) {
            const int64_t q = e / kOut;
            const int c = (int)(e - q * kOut);
            double s = 0.0;
            for (int sp = 0; sp < pl.b; ++sp) s += __ldcg(args.partial + ((int64_t)sp * m + q) * kOut + c);
            put_result(args, ra, rj, rs, q, c, s);
        }
    } else {
        // Many chunks (small blocks): one warp per (particle, value); lane l
        // sums chunks l, l+32, ..., then a fixed butterfly combines the lanes.
        // Consecutive (particle, value) pairs go to warps of different CTAs, so
        // that a small block's few sums run on as many FP64 units (one per
        // scheduler, ~64 cycles per warp instruction) as there are sums.
        const int lane = (int)(threadIdx.x & 31);
        const int64_t wid = (int64_t)blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5);
        const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
        for (int64_t e = wid; e < total; e += nw) {
            const int64_t q = e / kOut;
            const int c = (int)(e - q * kOut);
            double s = 0.0;
            for (int sp = lane; sp < pl.b; sp += 32) s += __ldcg(args.partial + ((int64_t)sp * m + q) * kOut + c);
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) put_result(args, ra, rj, rs, q, c, s);
        }
    }
}

__global__ void k_reduce(const EvalArgs args, double *ra, double *rj, double *rs)
{
    const int64_t m = args.m_dev ? *args.m_dev : args.m_host;
    if (m <= 0) return;
    const Plan pl = args.plan_dev ? *args.plan_dev : args.plan_host;
    reduce_values(args, m, pl, ra, rj, rs, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

template <class P, bool G>
cudaError_t set_attr()
{
    return cudaFuncSetAttribute(k_eval<P, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<P>());
}

template <class P, bool G>
int occupancy()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval<P, G>, kEvalThreads, smem_bytes<P>()) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace

cudaError_t eval_setup(int)
{
    cudaError_t e;
    if ((e = set_attr<MixedEval, false>()) != cudaSuccess) return e;
    if ((e = set_attr<MixedEval, true>()) != cudaSuccess) return e;
    if ((e = set_attr<F64, false>()) != cudaSuccess) return e;
    return set_attr<F64, true>();
}

int eval_grid(bool mixed, int num_sms)
{
    return (mixed ? occupancy<MixedEval, false>() : occupancy<F64, false>()) * num_sms;
}

namespace {
template <class P>
cudaError_t launch_one(const EvalArgs &args, int grid, cudaStream_t st)
{
    if (args.guard)
        k_eval<P, true><<<grid, kEvalThreads, smem_bytes<P>(), st>>>(args);
    else
        k_eval<P, false><<<grid, kEvalThreads, smem_bytes<P>(), st>>>(args);
    return cudaGetLastError();
}

template <class P>
int clip_grid(const EvalArgs &args, int num_sms)
{
    const int64_t full = (int64_t)occupancy<P, false>() * num_sms;
    if (args.plan_dev || args.bv.nc > 0) return (int)full;
    const int64_t items = args.plan_host.n_items;
    return (int)(items < full ? (items > 0 ? items : 1) : full);
}
}  // namespace

int eval_launches(bool, const EvalArgs &) { return 1; }

cudaError_t launch_eval(bool mixed, const EvalArgs &args, int num_sms, cudaStream_t st)
{
    if (!mixed) return launch_one<F64>(args, clip_grid<F64>(args, num_sms), st);
    return launch_one<MixedEval>(args, clip_grid<MixedEval>(args, num_sms), st);
}

cudaError_t launch_reduce(const EvalArgs &args, double *ra, double *rj, double *rs, int grid, cudaStream_t st)
{
    k_reduce<<<grid, 256, 0, st>>>(args, ra, rj, rs);
    return cudaGetLastError();
}

// Overheads in units of one thread's j-iteration (I interactions): per tile the
// barrier and the bulk-copy issue; per work item the pipeline fill, the lane
// reduction and the partial-sum stores.  The FP64 iteration is ~30x longer than
// the mixed one, so its per-item overhead is relatively small.
PlanParams plan_params(bool mixed, int64_t npad, int num_sms, int64_t pcap, int tpi_force, int b_force)
{
    PlanParams q;
    q.tj = mixed ? MixedEval::TJ : F64::TJ;
    q.i_per_thread = mixed ? MixedEval::I : F64::I;
    q.ntiles = npad / q.tj;
    q.pcap = pcap;
    q.grid = eval_grid(mixed, num_sms);
    q.tpi_force = tpi_force;
    q.b_force = b_force;
    q.c_tile = mixed ? 2 : 1;
    q.c_item = mixed ? 24 : 2;
    // One kernel per precision (the planner's second-variant fields unused).
    q.variants = 1;
    q.ipt1 = q.i_per_thread;
    q.grid1 = q.grid;
    q.weight1 = q.weight1_one = 100;
    for (int k = 0; k < kTuneBuckets; ++k) q.tuned[k] = -1;
    return q;
}

}  // namespace hg
