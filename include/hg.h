/*
 * hg.h -- C ABI of the GB300 (sm_103a) direct-summation engine for the
 * 6th-order Hermite block-timestep N-body method of Capuzzo-Dolcetta, Spera &
 * Punzo (HiGPUs, "A fully parallel, high precision, N-body code running on
 * hybrid computing platforms").
 *
 * Conventions shared by every call
 *  - Units: G = 1.  Indices are 0-based int32.  Vectors are [n][3] row-major
 *    doubles (x, y, z of particle 0, then particle 1, ...).
 *  - Pointer arguments may point to host memory or to device memory of the
 *    context's GPU; the library tells them apart with cudaPointerGetAttributes.
 *    The caller owns every pointer it passes and may reuse it when the call
 *    returns: inputs are copied, outputs are written before the return.
 *  - Every call runs on the context's CUDA stream (hg_opts.stream, else a
 *    stream the context creates).  Calls that return values in host memory
 *    synchronize that stream; the others only enqueue work.
 *  - Every int-returning call returns HG_OK (0) or one of the HG_E* codes;
 *    hg_last_error() then holds a message.  A failed call leaves the
 *    integration state as it was, except HG_ECUDA and HG_ETIMEOUT, after which
 *    the context should be freed.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef HG_H
#define HG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HG_OK 0
#define HG_EINVAL 1     /* bad argument (size, pointer, value, order of indices) */
#define HG_ENOMEM 2     /* device or host allocation failed */
#define HG_ECUDA 3      /* a CUDA call failed */
#define HG_ESTATE 4     /* call out of order, or particle not due at the block time */
#define HG_ETIMEOUT 5   /* a bounded device-side wait expired; results are invalid */

#define HG_FP64 0       /* FP64 pair arithmetic and FP64 sums */
#define HG_MIXED 1      /* FP32 pair arithmetic (two pairs per packed f32x2 instruction),
                           double-single position differences, compensated FP32 sums
                           widened to FP64; FP64 state and corrector.  The step criterion
                           may not shrink a step whose 4th-order residual lies below
                           3e-6 sum_j m_j / (r_ij^2 + eps^2), the evaluation's noise scale */

typedef struct hg_ctx hg_ctx;

/* Options.  Fill with hg_default_opts() and change what you need. */
typedef struct hg_opts {
    int32_t precision;        /* HG_FP64 or HG_MIXED for the acc/jerk/snap evaluation */
    int32_t energy_precision; /* HG_FP64 or HG_MIXED pair arithmetic inside hg_energy */
    int32_t device;           /* CUDA device ordinal */
    int32_t tpi;              /* 0 = automatic, else threads sharing one i-particle (1..64, power of 2) */
    int32_t jsplit;           /* 0 = automatic, else number of j-chunks per i-tile ("Bfactor") */
    int32_t graph_steps;      /* block steps captured per CUDA graph in hg_step/hg_advance (default 8) */
    int32_t start_mode;       /* 0 = start-up evaluation in hg_init (default); 1 = none: acc, jerk, snap,
                                 crackle and t are zero and dt = dt_max until hg_set_state (resume) */
    int32_t profile;          /* 1 = time the sections of every graph-replayed block step with CUDA
                                 events (hg_get_profile); adds a synchronization per graph replay */
    int32_t test_stall_eval;  /* testing only: 1 = every evaluation expects bytes that are never
                                 copied, so its bounded waits run out (~2 s) and the call returns
                                 HG_ETIMEOUT; exercises the failure path without a fault */
    int32_t order;            /* integration order: 6 (default; 0 also means 6) is the paper's 6th-order
                                 Hermite scheme; 4 is the 4th-order Hermite scheme its step criterion
                                 admits with p = 4 (corrector from a and jerk, snap and crackle from the
                                 cubic interpolant; stored snap and crackle stay zero) */
    double dt_min;            /* smallest step, power of two (default 2^-25, Sect. 3) */
    double dt_max;            /* largest step, power of two (default 2^-3, Sect. 3) */
    double eta_init;          /* accuracy parameter of the first step (p = 4 criterion; default 0.01) */
    void *stream;             /* cudaStream_t to run on; NULL = the context creates one */
} hg_opts;

/* The state of every particle at its own time t_i (Sect. 3: r, v, a, jerk, snap,
 * crackle, individual step).  Caller-allocated arrays of n or [n][3] doubles,
 * host or device.  t_sys is the last block time the system reached. */
typedef struct hg_state {
    double *mass;     /* [n] */
    double *pos;      /* [n][3] */
    double *vel;      /* [n][3] */
    double *acc;      /* [n][3] */
    double *jerk;     /* [n][3] */
    double *snap;     /* [n][3] */
    double *crackle;  /* [n][3] */
    double *t;        /* [n] */
    double *dt;       /* [n] power-of-two steps */
    double t_sys;
} hg_state;

/* Counters kept on the device. */
typedef struct hg_stats {
    int64_t block_steps;   /* block steps taken by hg_step/hg_advance */
    int64_t interactions;  /* sum over those steps of m * n (pair evaluations incl. j == i) */
    int64_t last_m;        /* size of the last block */
    double t_sys;          /* last block time */
    int64_t kernels;       /* kernel launches issued by the library (graph replays count every node) */
} hg_stats;

/* Device time of the block-step sections (Table 1: next-block selection,
 * prediction, evaluation, j-split reduction, correction), accumulated over the
 * graph-replayed block steps taken with opts.profile = 1. */
typedef struct hg_profile {
    double ms[5];          /* next, predict, evaluate, reduce, correct */
    int64_t block_steps;   /* block steps (including no-op steps past t_end) timed */
} hg_profile;

/* Fill opts with the defaults listed above. */
void hg_default_opts(hg_opts *opts);

/* Create a context for n particles (masses [n] > 0, positions and velocities
 * [n][3], finite), softening eps >= 0 (Sect. 2, softened potential) and
 * accuracy parameter eta > 0 of the generalized Aarseth criterion (Sect. 3).
 * Performs the start-up: a full evaluation with every particle active at t = 0,
 * crackle = 0, first steps from the p = 4 criterion with opts->eta_init,
 * quantized to powers of two in [dt_min, dt_max].  opts may be NULL.
 * With eps = 0 particles at the same position exert no force on each other.
 * Value limits (HG_EINVAL beyond them), the ranges the pair arithmetic keeps
 * finite in: mixed |positions| <= 1e15, |velocities| <= 1e30, FP64 both 1e150;
 * eps at most the position limit; every mass <= L min(1, eps^3) with L = 1e37
 * (mixed) or 1e300 (FP64), only <= L with eps = 0, so that m / (r^2 + eps^2)
 * and m / (r^2 + eps^2)^(3/2) stay finite for every pair.  hg_set_state and hg_bind_device check the same limits (and
 * 1e30 / 1e150 for the higher derivatives).
 * Errors: HG_EINVAL, HG_ENOMEM, HG_ECUDA. */
int hg_init(hg_ctx **out, int64_t n, const double *mass, const double *pos, const double *vel,
            double eps, double eta, const hg_opts *opts);

/* Independent clusters in one context: particles [offsets[c], offsets[c+1]) of
 * the concatenated arrays form cluster c (offsets: n_clusters + 1 int64, host
 * or device, offsets[0] = 0, offsets[n_clusters] = n, every cluster non-empty).
 * A particle feels only its own cluster; each cluster keeps its own block-time
 * hierarchy while all clusters advance together in global block steps (every
 * particle due at the global next block time is active), evaluated in one
 * persistent kernel per block step.  Every other call works on the whole set;
 * hg_energy returns sums over clusters of each cluster's own K and W (FP64
 * pairs).  n_clusters = 0 is hg_init.  Errors as hg_init. */
int hg_init_batch(hg_ctx **out, int32_t n_clusters, const int64_t *offsets, int64_t n, const double *mass,
                  const double *pos, const double *vel, double eps, double eta, const hg_opts *opts);

/* Table 1, section 1: t_next = min_i (t_i + dt_i) and the ascending indices of
 * the m particles with t_i + dt_i == t_next.  Makes them the context's current
 * block.  idx (host or device, capacity cap) receives the list when non-NULL;
 * a list longer than cap gives HG_EINVAL with *m_out still set. */
int hg_next_block(hg_ctx *ctx, double *t_next, int32_t *idx, int64_t cap, int64_t *m_out);

/* Sect. 3 item 1: predict positions, velocities and accelerations of all n
 * particles to time t (Taylor series through crackle), in FP64. */
int hg_predict(hg_ctx *ctx, double t);

/* Sect. 3 item 2: acceleration, jerk and snap of the m listed particles from
 * all n predicted particles (direct sum, j != i, softened), in the context's
 * precision.  idx: strictly increasing, in range, host or device; NULL = the
 * current block of hg_next_block (then m must equal its size).  acc, jerk,
 * snap: [m][3] outputs (host or device) or NULL to keep the results on the
 * device for hg_correct.  Needs a preceding hg_predict.  Errors: HG_EINVAL,
 * HG_ESTATE (no prediction), HG_ECUDA, HG_ETIMEOUT. */
int hg_evaluate(hg_ctx *ctx, const int32_t *idx, int64_t m, double *acc, double *jerk, double *snap);

/* The condition scale of the last hg_evaluate of a mixed context: for each of
 * its m particles (in the order of its list), sum_{j != i} m_j / (r_ij^2 +
 * eps^2) over the predicted data, summed in FP32 like the evaluation (an upper
 * bound of sum_j |a_ij|, equal to it for r_ij >> eps).  FP32 rounding of the
 * pair terms errs in a_i in proportion to it, so scale_i / |a_i| is the
 * particle's condition number; the step criterion's noise floor uses it too.
 * out: [m] doubles, host or device.  Errors: HG_ESTATE (FP64 context, or no
 * pending evaluation), HG_EINVAL (m differs from the evaluation's).
 * Synchronizes.  (The paper has no counterpart: its hybrid precision has no
 * noise analysis.) */
int hg_condition_scale(hg_ctx *ctx, double *out, int64_t m);

/* Sect. 3 item 3 and the time-step update: correct the particles of the last
 * hg_evaluate (idx NULL, or the same list), derive crackle from the Hermite
 * interpolant, take the new step from the p = 6 criterion quantized to powers
 * of two, and advance their time to the prediction time.  Every listed particle
 * must satisfy t_i + dt_i == prediction time (HG_ESTATE otherwise). */
int hg_correct(hg_ctx *ctx, const int32_t *idx, int64_t m);

/* n_steps complete block steps (next block, predict, evaluate, j-split
 * reduction, correct), entirely on the device and replayed from CUDA graphs;
 * no host synchronization inside.  Errors: HG_EINVAL, HG_ECUDA. */
int hg_step(hg_ctx *ctx, int64_t n_steps);

/* Block steps until the next block time would exceed t_end (choose t_end a
 * multiple of dt_max to end with every particle at t_end).  *steps_out, if
 * non-NULL, receives the number of block steps taken.  Graphs of graph_steps
 * block steps are replayed with the next one queued while the host reads the
 * previous one's stop flag, so up to one graph of empty steps (m = 0, every
 * kernel returns at once) runs past t_end; they change nothing and are not
 * counted as block steps.  Synchronizes. */
int hg_advance(hg_ctx *ctx, double t_end, int64_t *steps_out);

/* Kinetic and potential energy (Sect. 2 softened potential, W = -sum_{i<j}
 * m_i m_j / sqrt(r^2 + eps^2)) of the system predicted to the last block time,
 * summed in FP64 (pair arithmetic per opts.energy_precision).  Uses its own
 * buffers: a pending hg_predict/hg_evaluate stays valid.  Synchronizes. */
int hg_energy(hg_ctx *ctx, double *kinetic, double *potential);

/* Total angular momentum L = sum_i m_i r_i x v_i (L[3], host) of the system
 * predicted to the last block time, summed in FP64 in a fixed order: the
 * quantity whose magnitude Sect. 5.1 follows for conservation.  Uses its own
 * buffers like hg_energy.  Synchronizes. */
int hg_angular_momentum(hg_ctx *ctx, double *L);

/* Copy the state out (every non-NULL field) / replace it (every field required).
 * hg_set_state checks: masses > 0, finite values, dt a power of two in
 * [dt_min, dt_max], t_i >= 0 and a multiple of dt_i; it invalidates any
 * prediction. */
int hg_get_state(hg_ctx *ctx, hg_state *out);
int hg_set_state(hg_ctx *ctx, const hg_state *in);

/* Bind caller-owned device arrays (e.g. torch tensors) as the context's state:
 * dev's nine arrays (n or [n][3] doubles each, device memory of the context's
 * GPU, 8-byte aligned; t_sys is ignored) replace the context's own, so the
 * caller reads and writes the state in place.  copy_in != 0 first copies the
 * current state into them; copy_in = 0 takes what they hold, which must pass the
 * checks of hg_set_state (HG_EINVAL otherwise, nothing bound).  dev = NULL
 * unbinds: the state is copied back into the context's own arrays.  The caller
 * keeps the arrays alive while bound (hg_free never frees them) and touches
 * them only when the context's stream is idle (after a synchronizing call, or
 * ordered on that stream).  The captured graphs are rebuilt on their next use.
 * (The binding is a library convenience; the paper has no counterpart.) */
int hg_bind_device(hg_ctx *ctx, const hg_state *dev, int copy_in);

/* Device counters (synchronizes). */
int hg_get_stats(hg_ctx *ctx, hg_stats *out);

/* Section times accumulated so far (zeros unless opts.profile = 1); reset != 0
 * clears them after the copy. */
int hg_get_profile(hg_ctx *ctx, hg_profile *out, int reset);

/* Number of particles of the context. */
int64_t hg_size(const hg_ctx *ctx);

/* Message of the last failed call on ctx (never NULL; "" if none).  Owned by ctx. */
const char *hg_last_error(const hg_ctx *ctx);

/* Message of the last failed hg_init or hg_evaluate_static on this thread
 * (calls that have no context to hold it). */
const char *hg_init_error(void);

/* An evaluation that allocates no memory, for callers that must not call
 * cudaMalloc: code running inside a host application or framework that owns
 * all device memory through its own pool or arena, or that has fixed its device
 * memory budget at start-up, or whose work must not be interrupted by the device
 * synchronization an allocation can cause.  (The paper has no counterpart; it
 * is a library convenience.)  Computes acc, jerk and snap of the m listed
 * particles like hg_evaluate, without a context: the caller passes predicted
 * data directly.
 *   n          particles, 1 <= n <= 16384 (larger n: HG_EINVAL);
 *   mass       [n], pos, vel, acc_pred [n][3]: predicted masses, positions,
 *              velocities and accelerations, FP64, device memory, within the
 *              limits hg_init checks (not checked here: values beyond them give
 *              non-finite results);
 *   eps        softening >= 0; precision HG_FP64 or HG_MIXED;
 *   idx        [m] device int32, strictly increasing, in [0, n) (HG_EINVAL otherwise);
 *   acc, jerk, snap  [m][3] FP64 device outputs; stream  cudaStream_t or NULL.
 * Its scratch is one fixed array of about 6.5 MB in the library's device
 * memory, kept on a device until the process exits once it is there.  The
 * first call on a device (any m) looks up that array's address; under CUDA's
 * default lazy module loading that first call is also when the driver loads
 * the array onto the device, i.e. allocates its 6.5 MB (set
 * CUDA_MODULE_LOADING=EAGER to have it allocated when the library is loaded
 * instead).  A call with m = 0 does only this set-up: make one at start-up,
 * before any stream capture on that device, so that later calls allocate
 * nothing.  Every call shares the array, so calls whose work overlaps on the
 * GPU (different streams or threads) race; the call synchronizes its stream
 * before returning.  Errors as hg_evaluate, message in hg_init_error(). */
int hg_evaluate_static(int64_t n, const double *mass, const double *pos, const double *vel, const double *acc_pred,
                       double eps, int32_t precision, const int32_t *idx, int64_t m, double *acc, double *jerk,
                       double *snap, void *stream);

/* Measured arithmetic peak of the CUDA cores of `device`, the denominator of
 * the evaluation kernels' roofline (the paper derives its peaks from unit
 * counts and clock, Sect. 5.7 and Table 2; this measures them).  form: 0 =
 * scalar FP32 FMA, 1 = packed FP32 FMA (fma.rn.f32x2, the mixed evaluation's
 * form), 2 = FP64 FMA.  Every SM is filled with threads that each advance 8
 * independent FMA chains; one warm-up launch, then one launch timed with CUDA
 * events on `stream` (cudaStream_t or NULL).  *tflops receives the FMA rate in
 * TFLOP/s (2 flops per FMA and lane), *ms (may be NULL) the timed launch's
 * duration.  Changes no device setting (clocks stay as they are: the figure is
 * taken at whatever clock the GPU runs).  Allocates 16 bytes for the duration
 * of the call.  Errors: HG_EINVAL (form, device), HG_ECUDA; message in
 * hg_init_error().  Synchronizes. */
int hg_peak_flops(int32_t form, int32_t device, void *stream, double *tflops, double *ms);

/* ------------------------------------------------------------------------
 * Autotuning of the evaluation's launch plan (the paper's "Bfactor", Sect. 3:
 * how the m active particles and the n j-particles are spread over the GPU).
 * Block sizes are grouped in HG_TUNE_BUCKETS buckets, bucket k holding
 * 2^k <= m < 2^(k+1).  For each bucket the table holds -1 (use the built-in
 * cost model) or a measured choice:
 *  - one system: a plan index k in [0, 224): 2^(k / 32) threads share one
 *    i-particle and each j-chunk holds T[k % 32] j-tiles (256 records mixed,
 *    128 FP64), T = {1, 2, ..., 16, 20, 24, 32, 40, 48, 64, 96, 128, 192, 256,
 *    384, 512, 1024, 2048, 4096, 8192}.  Both kernels hold one i-particle per
 *    thread, so the i-tile is 128 / 2^(k/32) particles;
 *  - clusters (hg_init_batch): a code w + 8 (s + 1), w in [0, 6], s in
 *    {-1, 0, 1}: the j-split is the largest one leaving at least 2^w work items
 *    per resident CTA, and each cluster's threads per i-particle are 2^s times
 *    the number that fills one CTA with its active particles.
 * A plan that is not admissible for the actual m (partial-sum capacity, or the
 * opts.tpi / opts.jsplit overrides) falls back to the cost model.
 * ------------------------------------------------------------------------ */
#define HG_TUNE_BUCKETS 32

/* One bucket measured by hg_tune. */
typedef struct hg_tune_entry {
    int64_t m;           /* middle block size timed (the m particles with the smallest steps) */
    int32_t bucket;      /* floor(log2 m) */
    int32_t candidates;  /* plans timed */
    int32_t model;       /* the cost model's choice, in table encoding */
    int32_t chosen;      /* value stored in the table (-1: the cost model was kept) */
    double model_us;     /* device time of evaluation + reduction with the model's plan, us */
    double best_us;      /* the same for the stored choice (model_us when chosen == -1) */
} hg_tune_entry;

/* Measure, for every bucket whose m is at most m_max (0: n; the m of bucket k is
 * 1 for k = 0 and 1.5 * 2^k clamped to n above), the cost model's plan and its
 * cheapest rivals on the context's current predicted data, with CUDA events on
 * the context's stream, each plan launched reps times (0: automatic) after one
 * warm-up.  Because one stored plan serves the whole bucket, every plan is timed
 * at the bucket's block sizes 2 and 3 (k = 1) or 2^k * 5/4, 3/2 and 7/4 (k >= 2),
 * clamped to n, and the times are summed; a rival is stored only if its sum is
 * at least 3% below the cost model's.  model_us and best_us report the mean
 * over those block sizes.  The
 * integration state is unchanged, a pending hg_evaluate is dropped and the
 * captured graphs are rebuilt on their next use.  report (capacity cap, may be
 * NULL) receives one entry per bucket measured; *n_out their number.
 * Errors: HG_EINVAL, HG_ECUDA, HG_ETIMEOUT.  Synchronizes. */
int hg_tune(hg_ctx *ctx, int64_t m_max, int32_t reps, hg_tune_entry *report, int32_t cap, int32_t *n_out);

/* Device time of one evaluation (evaluation and j-split reduction kernels,
 * with the launch plan the context would choose for m: tuning table, else cost
 * model, subject to opts.tpi / opts.jsplit) of the m listed particles (idx
 * strictly increasing, in range, host or device) against the data of the last
 * hg_predict: one warm-up launch, then reps launches (0: automatic, ~2 ms
 * worth, 3 to 64) timed with CUDA events on the context's stream; *us receives
 * the mean in microseconds.  The integration state is unchanged; the results
 * are not kept (a pending hg_evaluate is dropped, the prediction stays).  The
 * measurement the tuner makes, offered for benchmarks such as the paper's
 * Bfactor comparison (Sect. 5.5).  Errors: HG_EINVAL, HG_ESTATE (no
 * prediction), HG_ECUDA, HG_ETIMEOUT.  Synchronizes. */
int hg_time_evaluate(hg_ctx *ctx, const int32_t *idx, int64_t m, int32_t reps, double *us);

/* Copy the tuning table out / replace it (HG_TUNE_BUCKETS int16 values, host
 * memory; -1 entries use the cost model).  hg_set_tuning checks every value for
 * the context's kind (HG_EINVAL otherwise), so a table saved from one context
 * can be given to another of the same precision and kind on the same GPU model. */
int hg_get_tuning(hg_ctx *ctx, int16_t *table);
int hg_set_tuning(hg_ctx *ctx, const int16_t *table);

/* Host-side fault injection, for testing the failure paths without a device
 * fault (the library convenience has no counterpart in the paper).  After
 * hg_inject_fault(HG_FAULT_ALLOC, n) the n-th device allocation the library
 * makes for a context fails as if cudaMalloc had (the call returns HG_ENOMEM);
 * after hg_inject_fault(HG_FAULT_CUDA, n) the n-th CUDA runtime call a
 * context-based call checks fails without being made (HG_ECUDA, message
 * "injected fault").  One fault, then the injector disarms itself;
 * HG_FAULT_NONE disarms it.  Process-wide, counted across threads.  The
 * environment variable HG_FAULT=alloc:<n> or HG_FAULT=cuda:<n> arms it when
 * the library is loaded.  Errors: HG_EINVAL (kind, or n < 1). */
#define HG_FAULT_NONE 0
#define HG_FAULT_ALLOC 1
#define HG_FAULT_CUDA 2
int hg_inject_fault(int32_t kind, int64_t nth);

/* The checked build (compiled with -DHG_CHECKED, paper_1207_2367_gb300/_lib/
 * libhgpu_checked.so) adds device bounds checks on every active-list entry,
 * j-tile range and partial-sum row the evaluation, reduction and correction
 * kernels touch: a value out of range is not used (the access is skipped or
 * clamped) and the next synchronizing call returns HG_ECUDA with a message,
 * instead of a memory fault.  hg_build_checked() returns 1 in that build, 0 in
 * the normal one.  Testing only: hg_test_corrupt_list writes value into entry
 * pos of the context's current block list (after hg_next_block), so that the
 * checks can be seen to fire; the normal build refuses it (HG_EINVAL) and
 * touches nothing.  (Library conveniences; the paper has no counterpart.) */
int hg_build_checked(void);
int hg_test_corrupt_list(hg_ctx *ctx, int64_t pos, int32_t value);

/* Release the context and its device memory.  NULL is allowed. */
void hg_free(hg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HG_H */
