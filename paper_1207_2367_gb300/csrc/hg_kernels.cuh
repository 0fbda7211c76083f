// hg_kernels.cuh -- launchers of the FP64 block-step kernels (hg_kernels.cu).
#pragma once

#include "hg_internal.cuh"

namespace hg {

struct StepParams {
    double eta, eta_init, dt_min, dt_max;
    // Relative noise floor of the evaluated acceleration (0: exact enough, FP64).
    // When |a1 - a0 - j0 h - s0 h^2/2| < noise_rel * scale (the evaluation's
    // noise scale sum_j m_j / r_ij^2, else |a1|) the interpolated crackle, pop
    // and 5th derivative are unresolved: the criterion then does not shrink the step.
    double noise_rel;
    float log2_eta;   // log2(eta), for the FP32 estimate of the criterion
    int order;        // 6: the paper's scheme (p = 6); 4: the 4th-order scheme (p = 4)
};

constexpr int64_t kNBChunk = 2048;   // particles per CTA in the next-block passes

int nb_grid(int64_t n);
// part, cnt, off: nb_grid(n) entries each.
cudaError_t launch_next_block(const State &st, int64_t n, double *part, int32_t *cnt, int32_t *off, int32_t *idx,
                              DevScalars *sc, int count_step, const PlanParams &pq, cudaStream_t s);
// Pass 1 alone: sc->tnext_bits = bits of min_i tend_i.
cudaError_t launch_next_min(const State &st, int64_t n, double *part, DevScalars *sc, cudaStream_t s);
// One system, graph-replayed block steps: block selection fused into the
// prediction.  Needs sc->tnext_bits = min_i tend_i (kept by launch_correct with
// min_pass); predicts every record to t_next, lists the due particles in idx
// (arbitrary order), sets m, t_cur, done, the counters and the plan.
cudaError_t launch_predict_select(bool mixed, const State &st, const Records &rec, int64_t n, int64_t npad,
                                  int32_t *idx, DevScalars *sc, int count_step, const PlanParams &pq, int max_grid,
                                  cudaStream_t s);
// After the state was replaced: tend = t + dt and the FP32 copies (st.f32).
cudaError_t launch_tend(const State &st, int64_t n, cudaStream_t s);
// The FP32 copies alone (a no-op for FP64 contexts, st.f32 == nullptr).
cudaError_t launch_f32(const State &st, int64_t n, cudaStream_t s);
// rmap: record of each particle (clusters), or nullptr (record i = particle i).
cudaError_t launch_predict(bool mixed, const State &st, const Records &rec, int64_t n, int64_t npad,
                           const double *t_dev, double t_host, const int64_t *m_dev, const int32_t *rmap,
                           cudaStream_t s);
// Clusters in a block step: predict only the clusters with active particles
// (after the batch planning kernel of that step).
cudaError_t launch_predict_clusters(bool mixed, const State &st, const Records &rec, int64_t n, const BatchView &bv,
                                    const double *t_dev, const int64_t *m_dev, cudaStream_t s);
// Padding in every record slot (cluster contexts, before the first prediction).
cudaError_t launch_pad_records(bool mixed, const Records &rec, int64_t npad, cudaStream_t s);
// Work list of one evaluation over clusters (sizes on the device or host), with
// the knobs of q.tuned for the block's size; count != nullptr adds the step's
// pair evaluations to count->interactions.
cudaError_t launch_batch_plan(const int32_t *idx, const int64_t *m_dev, int64_t m_host, const BatchView &bv,
                              const PlanParams &q, DevScalars *count, cudaStream_t s);
cudaError_t launch_start(const State &st, int64_t n, const double *ra, const double *rj, const double *rs,
                         const StepParams &sp, cudaStream_t s);
// Corrector and new steps of the listed particles.  min_pass (graph steps of
// one system, where the list is every particle due at sc->t_cur): also leave
// min_i tend_i of the new state in sc->tnext_bits (reset beforehand by the
// selection).  rn: noise scale of each listed particle (mixed), or nullptr
// (the noise floor then scales with |a1|).  grid: CTAs of 128 threads.
cudaError_t launch_correct(const State &st, const int32_t *idx, const int64_t *m_dev, int64_t m_host, int64_t n,
                           const double *ra, const double *rj, const double *rs, const double *rn,
                           const StepParams &sp, DevScalars *sc, int min_pass, int grid, cudaStream_t s);
int energy_splits(int64_t n, int num_sms);
cudaError_t launch_energy(bool mixed, const State &st, int64_t n, double t, double eps2, double *xe, double *ve,
                          double *phi_part, int nsplit, double *part2, int g2, double *out2, const BatchView &bv,
                          cudaStream_t s);
// L = sum_i m_i r_i x v_i of the system predicted to t, into out3 (part3: 3 g doubles).
cudaError_t launch_angular_momentum(const State &st, int64_t n, double t, double *xe, double *ve, double *part3,
                                    int g, double *out3, cudaStream_t s);
// Largest magnitudes a state may hold: pos for positions, deriv for velocities
// and the higher derivatives (a value beyond them, or not finite, is refused).
// The mixed path's FP32 pair arithmetic squares position differences and forms
// products of derivatives and differences, so its limits keep those in FP32's
// range; the FP64 path's keep them in FP64's.
// mass bounds the masses and the pair law's largest factors: every pair, the one
// of a particle with itself included, has m_j / (r^2 + eps^2)^(3/2) <= m_j / eps^3
// and m_j / (r^2 + eps^2) <= m_j / eps^2, kept below L = 1e37 in the mixed path
// (FLT_MAX is 3.4e38) and L = 1e300 in the FP64 path by m <= L min(1, eps^3).
// With eps = 0 the pairs at r = 0 are skipped and only m <= L applies.
struct ValueLimits {
    double pos, deriv, mass;
};
inline ValueLimits value_limits(bool mixed, double eps)
{
    const double L = mixed ? 1e37 : 1e300;
    const double e3 = eps * eps * eps;
    const double mass = eps > 0.0 && e3 < 1.0 ? L * e3 : L;
    return mixed ? ValueLimits{1e15, 1e30, mass} : ValueLimits{1e150, 1e150, mass};
}
// eps^2 below this (or eps = 0) selects the evaluation that skips pairs whose
// softened r^2 is zero: FP32 rounds such an eps^2 to zero.
constexpr double kGuardEps2 = 0x1p-100;
cudaError_t launch_validate_init(const double *mass, const double *x, const double *v, int64_t n,
                                 const ValueLimits &lim, int32_t *flag, cudaStream_t s);
cudaError_t launch_validate_state(const State &st, int64_t n, double dt_min, double dt_max, const ValueLimits &lim,
                                  int32_t *flag, cudaStream_t s);
cudaError_t launch_validate_idx(const int32_t *idx, int64_t m, int64_t n, int32_t *flag, cudaStream_t s);
cudaError_t launch_check_correct(const State &st, const int32_t *given, const int32_t *cur, int64_t m, int64_t n,
                                 double t_pred, int32_t *flag, cudaStream_t s);

}  // namespace hg
