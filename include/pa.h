/*
 * pa.h -- C ABI of the GB300 (sm_103a) population-annealing library for the 2D Ising
 * ferromagnet (J = 1, L x L periodic lattice), after Weigel, Barash, Shchur and Janke,
 * "Understanding population annealing Monte Carlo simulations", arXiv:2102.06611.
 *
 * The entry points follow the method's step list (Sec. II):
 *   pa_init        step 1  simple sampling of R replicas at beta_0 = 0, then measurement
 *   pa_resample    step 2  reweighting by exp(-(beta_i - beta_{i-1}) E_j), Eq. (Q) for
 *                          Q_i, Eq. (taus) for the rescaled copy means, Eq.
 *                          (resampling-factors) or Poisson copy numbers, replica copying
 *   pa_anneal_step step 3  theta Metropolis sweeps of every replica, then measurement
 *   pa_observables step 4  population averages (Sec. III) and the free-energy estimator
 *                          Eq. (free-emergy-estimator) with ln Z_0 = L^2 ln 2 (Sec. VII)
 *
 * Memory: the library never allocates device memory.  The caller allocates every device
 * buffer (sizes from pa_query_sizes) and keeps it alive until pa_destroy.  The context
 * object itself is host memory owned by the library.
 *
 * Streams: every call is asynchronous on the stream given to pa_init, except the calls
 * documented as synchronising (they copy results to host memory).
 *
 * Errors: every call returns a pa_status.  Kernels never trap: a device-side failure
 * (population above capacity, extinct population) sets a sticky error word that the next
 * synchronising call returns; after any error the context is only valid for
 * pa_last_error and pa_destroy.
 *
 * Random numbers are Philox4x32-10 (Salmon et al., SC'11) with key = seed and counters
 * keyed by (stream tag, step, sweep, replica slot, site), so every result is a fixed
 * function of (config, schedule) and does not depend on the launch configuration.
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pa_ctx pa_ctx;

typedef enum {
    PA_OK = 0,
    PA_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment, or unsupported L */
    PA_ERR_STATE = 2,       /* call out of order (e.g. resample to a lower beta) */
    PA_ERR_CAPACITY = 3,    /* resampled population larger than the buffer capacity */
    PA_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    PA_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    PA_ERR_NUMERIC = 6,     /* empty population or non-finite weights */
    PA_ERR_TOO_LARGE = 7    /* size above the fixed maximum of pa_copy_numbers_static */
} pa_status;

typedef enum {
    PA_RESAMPLE_NEAREST = 0,    /* Eq. (resampling-factors): floor(tau) or floor(tau) + 1 */
    PA_RESAMPLE_POISSON = 1,    /* r_j ~ Poisson(tau_hat_j), fluctuating population size */
    PA_RESAMPLE_MULTINOMIAL = 2 /* R children drawn from the parents with probabilities
                                   tau_j / R_{i-1} (Sec. II; fixed size R_i = R): integer
                                   weights W_j = floor(w_j 2^32), their exact running sum C_j,
                                   child c takes X = words 1:0 of Philox(ctr = (c, 0,
                                   MULTINOMIAL << 28, i)), U = floor(X C_last / 2^64), parent
                                   j with C_{j-1} <= U < C_j.  Single runs only. */
} pa_resample_kind;

/* Spin update of step 3 (Sec. IV).  With a aligned neighbours, dE = 4a - 8 and x the site's
   uniform 32-bit integer:
     Metropolis  a <= 2 flips; a = 3, 4 flip iff x < floor(e^{-beta dE} 2^32);
     heatbath    flip iff x < T_a, T_3 = floor(2^32 / (1 + e^{4 beta})),
                 T_4 = floor(2^32 / (1 + e^{8 beta})), T_1 = 2^32 - T_3, T_0 = 2^32 - T_4,
                 T_2 = 2^31 (flip probability 1 / (1 + e^{beta dE}) to 2^-32). */
typedef enum {
    PA_UPDATE_METROPOLIS = 0,
    PA_UPDATE_HEATBATH = 1
} pa_update_kind;

/* Run configuration.  L even, 4 <= L <= 128 (periodic L x L lattice).  The sizes 4, 8, 12,
   16, 20, 24, 32, 40, 48, 64, 80, 96 and 128 run kernels that hold a replica in registers;
   every other even L runs a kernel that stages it in shared memory (same random numbers and
   decisions, slower).  Batches (pa_batch_init) take every even L as well (register kernels
   for 4, 8, 12, 16, 24, 32, 48, 64 and 128, the shared-memory form for the others).
   1 <= R <= capacity <= 2^31 - 1.  beta_0 is always 0 (simple sampling, Sec. II). */
typedef struct {
    int L;
    int resample;                /* pa_resample_kind */
    long long R;                 /* target population size R (Eq. taus) */
    long long capacity;          /* replicas each buffer can hold (>= R) */
    unsigned long long seed;     /* Philox key */
    int update;                  /* pa_update_kind */
    int pad;                     /* 0 */
} pa_config;

/* Byte sizes of the caller-owned device buffers for a configuration.
   spin_bytes: one spin buffer (capacity * bytes_per_replica), 256-byte aligned start.
   int_bytes:  one per-replica int32 array (capacity * 4).
   work_bytes: the workspace. */
typedef struct {
    size_t spin_bytes;
    size_t int_bytes;
    size_t work_bytes;
    size_t bytes_per_replica;
} pa_sizes;

/* Caller-owned device buffers, each 256-byte aligned.  spins/level/mag/fam come in two
   copies (current population and resampling target). */
typedef struct {
    void *spins[2];
    void *level[2];   /* int32 energy level k = (E + 2N) / 4 per replica */
    void *mag[2];     /* int32 magnetisation M per replica */
    void *fam[2];     /* int32 family id (index of the beta_0 ancestor, Sec. V) */
    void *work;       /* workspace of pa_sizes.work_bytes */
} pa_buffers;

/* One record of step 4.  All floating-point fields are computed in binary64 in a fixed
   order from exact integer sums over the population.  Written by pa_observables and
   pa_record. */
typedef struct {
    long long step;        /* temperature index i (0 after pa_init) */
    long long R;           /* population size R_i */
    double beta;           /* beta_i */
    double dbeta;          /* beta_i - beta_{i-1} */
    double e;              /* energy per spin <E>/N                  (Sec. III) */
    double C;              /* specific heat per spin beta^2 Var(E)/N (Sec. III) */
    double m;              /* <|M|>/N                                (Sec. III) */
    double m2;             /* <M^2>/N^2 */
    double chi;            /* beta N (<M^2>/N^2 - m^2)               (Sec. III) */
    double lnQ;            /* ln Q_i of the last resampling          (Eq. Q) */
    double minus_betaF;    /* N ln 2 + sum_k ln Q_k                  (Sec. VII) */
    double rho_t;          /* R_i sum_k n_k^2, mean-square family size (Eq. rhot) */
    long long families;    /* number f of surviving families         (Sec. V) */
    long long sum_E;       /* exact integer sums the fields above are formed from */
    long long sum_E2;
    long long sum_absM;
    long long sum_M2;
    long long sum_size2;   /* sum over families of (family size)^2 */
    int theta;             /* sweeps of the last pa_anneal_step */
    int status;            /* sticky device error word (pa_status) */
    double sum_lnRratio;   /* sum_{k<=i} ln(R_{k-1} / R): the population-size factor of
                              Eq. modified-weights2 (0 at fixed population size) */
    long long R_target;    /* target population size R */
} pa_obs;

/* One temperature step of the schedule a context actually ran (see pa_schedule_log). */
typedef struct {
    long long step;        /* temperature index i */
    double beta;           /* beta_i */
    double dbeta;          /* beta_i - beta_{i-1} */
    double alpha;          /* histogram overlap of the proposal that produced beta_i (NaN if none) */
    int theta;             /* sweeps run at beta_i */
    int source;            /* PA_SCHED_* */
} pa_sched_entry;

enum {
    PA_SCHED_CALLER = 0,   /* beta_i passed by the caller */
    PA_SCHED_BISECT = 1,   /* from pa_propose_schedule (overlap bisection) */
    PA_SCHED_LEARNED = 2,  /* learned proposal accepted (overlap at or above the floor) */
    PA_SCHED_FALLBACK = 3  /* learned proposal rejected, bisection used instead */
};

/* Buffer sizes for cfg.  Returns PA_ERR_INVALID_ARG for an unsupported configuration. */
pa_status pa_query_sizes(const pa_config *cfg, pa_sizes *out);

/* Step 1 (Sec. II): create a context on `stream` (a cudaStream_t, NULL = legacy default
   stream) over the caller's buffers, fill R replicas by simple sampling at beta_0 = 0
   (site n of replica j is bit n mod 32 of word n/32 of Philox stream INIT), set family
   id j, and measure energies, magnetisations and the level histogram.  Asynchronous. */
pa_status pa_init(const pa_config *cfg, const pa_buffers *buf, void *stream, pa_ctx **out);

/* Step 2 (Sec. II, Eqs. Q, taus, resampling-factors): move from the current beta to
   beta_new >= beta.  Uses the energies measured before resampling (a population resampled
   again with no sweep in between is measured first); builds the level
   table in binary64 (w_k = exp(-dbeta (E_k - E_ref)), S = sum_k h_k w_k over the occupied
   levels in ascending k, in a fixed pairwise order: 1024 consecutive chunks, then a tree,
   tau_hat_k = R w_k / S), draws copy numbers, prefix-sums them on the device and copies
   children to consecutive slots in parent order (tree order).  Advances the step index.
   Asynchronous; a capacity overflow surfaces at the next synchronising call. */
pa_status pa_resample(pa_ctx *ctx, double beta_new);

/* Step 3 (Sec. II) and the measurement of step 4: theta >= 0 checkerboard Metropolis
   sweeps of every replica at the current beta (acceptance min(1, exp(-beta dE)) with
   integer thresholds floor(exp(-4 beta) 2^32), floor(exp(-8 beta) 2^32)), then
   energies, magnetisations and the level histogram.  Asynchronous. */
pa_status pa_anneal_step(pa_ctx *ctx, int theta);

/* Step 4: form a pa_obs record on the device and write it to `device_dst` (a device
   pointer to sizeof(pa_obs) bytes, 8-byte aligned).  Asynchronous. */
pa_status pa_record(pa_ctx *ctx, void *device_dst);

/* Step 4: form the record and copy it to host memory.  Synchronises the stream and
   returns the sticky device error, if any. */
pa_status pa_observables(pa_ctx *ctx, pa_obs *host_out);

/* Population analysis (Sec. IV, Eqs. neff, blocks, blocked_variance, jackknife-blocks,
   jackknife-variance; Sec. V, Eq. rhos).  The R_i replicas are taken in slot order, which
   is tree order (the children of one parent sit next to each other, so correlations are
   local), and cut into n contiguous blocks, block b = slots [floor(b R / n),
   floor((b + 1) R / n)).  From exact int64 block sums of E, E^2, |M|, M^2 every field below
   is formed in binary64 in a fixed order:
     var_X            unbiased variance of the unblocked series, (sum x^2 - R mean^2)/(R-1)
     var_mean_X_blocked   1/(n(n-1)) sum_b (X^B_b - mean_b X^B)^2, X^B_b = block mean
     var_mean_X_jack  (n-1)/n sum_b (X^J_b - mean_b X^J)^2, X^J_b = mean outside block b
     R_eff_X          var_X / var_mean_X_jack (effective number of independent replicas)
     var_C_jack       the same jackknife for C = beta^2 (<E^2> - <E>^2) / N
     S_f              -sum_k (s_k/R) ln(s_k/R) over families k of size s_k, summed by size
     rho_s            R / exp(S_f)
   for X = E (energy) and |M|. */
typedef struct {
    long long R;              /* population size R_i */
    long long families;       /* number of families f */
    int n_blocks;             /* n */
    int pad;
    double beta;              /* beta_i */
    double mean_E, var_E, var_mean_E_jack, var_mean_E_blocked, R_eff_E;
    double mean_absM, var_absM, var_mean_absM_jack, var_mean_absM_blocked, R_eff_M;
    double C, var_C_jack;
    double S_f, rho_s;
} pa_analysis;

/* Weighted average over M independent runs at one temperature step (Sec. VIII).  Run m's
   record gives R_i^m, R^m, -beta F^m and s^m = sum_k ln(R_{k-1}^m / R^m); the weights are
   omega_m proportional to R_i^m exp(-beta F^m) (mode 0, Eq. weighted-averages) or to
   R_i^m exp(s^m) exp(-beta F^m) (mode 1, Eq. modified-weights2), normalised in binary64 with
   the largest exponent taken out, runs in order.  Fields: the weighted and the plain means
   of e, C, m, m2, chi; M_eff = 1 / sum omega^2; the largest omega; the unbiased variance of
   -beta F^m over the runs (weighting is sound only while it is well below 1, Sec. VIII);
   and ln(sum_m R^m exp(-beta F^m) / sum_m R^m), the R-weighted mean of the runs' partition
   function estimates.  status = PA_ERR_INVALID_ARG if the records are not all at the same
   step and beta, else the first non-zero record status. */
typedef struct {
    long long step;
    int M;
    int mode;
    double beta;
    double M_eff, max_weight, var_minus_betaF, minus_betaF_combined;
    double e, C, m, m2, chi;                            /* weighted */
    double e_plain, C_plain, m_plain, m2_plain, chi_plain;
    int status;
    int pad;
} pa_weighted;

/* Form the weighted average of M >= 1 pa_obs records (device memory, contiguous, as written
   by pa_record or pa_batch_record) into *out_dev (device memory, sizeof(pa_weighted) bytes,
   8-byte aligned).  Asynchronous on `stream`; one block of one thread per call's result. */
pa_status pa_weighted_average(const void *records_dev, int M, int mode, void *out_dev, void *stream);

/* Analyse the current population (measured first if a resampling came since) in n_blocks
   blocks, 2 <= n_blocks <= min(R_i, 1024), and copy the result to host memory.
   Synchronising; PA_ERR_INVALID_ARG for a bad n_blocks (checked against R_i on the host). */
pa_status pa_analyze(pa_ctx *ctx, int n_blocks, pa_analysis *host_out);

/* Adaptive temperature step (the paper's self-adaptive steps, Sec. II; overlap guideline
   alpha > 0.7, Sec. X).  From the energy-level histogram h_k of the current population
   (measured at the current beta; measured first if a resampling came since), the overlap
   alpha(dbeta) = sum_k min(h_k / R, h_k w_k / S) of the energy distribution with its
   reweighting to beta + dbeta (w_k, S as in pa_resample) is evaluated in binary64 in a
   fixed order, and *beta_next receives beta + the largest dbeta in (0, hi],
   hi = min(dbeta_max, beta_final - beta), with alpha >= alpha_target (hi itself if it
   qualifies, else 48 bisection steps on [0, hi]; beta_final exactly when the whole
   remaining range qualifies).  *alpha_out receives alpha at that step.  Does not resample:
   pass *beta_next to pa_resample.  Synchronising.  0 < alpha_target <= 1, dbeta_max > 0,
   beta_final >= beta. */
pa_status pa_propose_schedule(pa_ctx *ctx, double alpha_target, double dbeta_max, double beta_final,
                              double *beta_next, double *alpha_out);

/* ---- Learned schedule.  The paper has no learned schedule: it names self-adaptive steps
   (Sec. II), advises alpha > 0.7 and an adaptive number of sweeps (Sec. X).  This is a design
   extension that only proposes; the overlap check below keeps every accepted step above a
   floor, and the schedule used is logged for exact replay.
   Network: 12 inputs -> 64 -> 64 -> 64 (tanh) -> 2 outputs, 9282 parameters in the flat
   order W1[64x12], b1[64], W2[64x64], b2[64], W3[64x64], b3[64], W4[2x64], b4[2] (row-major,
   W[out][in]), stored as bfloat16 bit patterns (uint16) for evaluation, float32 accumulation.
   Inputs (float32, from binary64 statistics of the current population): beta, ln L, ln R_i,
   <E>/N, ln(Var(E)/N + 1e-12), skewness and excess kurtosis of E, previous dbeta * L,
   previous theta / theta0, previous overlap, ln(rho_t) / ln(R_i) (Eq. rhot), fraction of
   parents given no copy at the last resampling.  Outputs (standardised): ln(dbeta sigma_E)
   (sigma_E = the population's energy standard deviation) and ln(theta). */
typedef struct {
    const unsigned short *params_bf16; /* device, 9282 bfloat16 patterns */
    const float *norm;                 /* device, 28 floats: x_mean[12], x_std[12], y_mean[2], y_std[2] */
} pa_learned_model;

typedef struct {
    double beta_next;   /* the step to pass to pa_resample */
    double alpha;       /* overlap at beta_next */
    double dbeta_prop;  /* the network's step before the check */
    int theta_next;     /* sweeps to run at beta_next (theta_prop if kept, theta0 on fallback) */
    int theta_prop;     /* the network's sweep count, clamped to [1, theta_max] */
    int source;         /* PA_SCHED_LEARNED or PA_SCHED_FALLBACK */
    int pad;
} pa_proposal;

/* Number of network parameters (9282). */
size_t pa_mlp_param_count(void);

/* Batched forward pass: y[batch x 2] from x[batch x 12]; act (optional, batch x 192 floats)
   receives the three hidden activations for pa_mlp_backward.  Asynchronous on `stream`. */
pa_status pa_mlp_forward(const unsigned short *params_bf16, const float *x, int batch, float *y, float *act,
                         void *stream);

/* Gradient of L = 1/(2 batch) sum (y - t)^2 with respect to the 9282 parameters (evaluated
   at their bfloat16 values) into grad (float32); delta is scratch of batch x 194 floats.
   Batch sums run in sample order (deterministic).  Asynchronous. */
pa_status pa_mlp_backward(const unsigned short *params_bf16, const float *x, const float *t, int batch,
                          const float *act, const float *y, float *delta, float *grad, void *stream);

/* One Adam step (Kingma & Ba) on float32 master parameters (step counts from 1), then the
   bfloat16 copy is refreshed by round-to-nearest-even.  Asynchronous. */
pa_status pa_mlp_adam(float *master, float *m, float *v, const float *grad, int step, float lr, float beta1,
                      float beta2, float eps, unsigned short *params_bf16, void *stream);

/* bfloat16 copy of float32 master parameters (round to nearest even).  Asynchronous. */
pa_status pa_mlp_round(const float *master, unsigned short *params_bf16, void *stream);

/* The 12 network inputs of the current population (measured first if needed) into
   host_out; previous-step inputs come from the context's schedule (theta0 scales theta).
   Synchronising. */
pa_status pa_features(pa_ctx *ctx, int theta0, float *host_out);

/* Learned step: features -> network -> (dbeta_prop, theta_prop) on the device; the step is
   kept if the overlap at min(dbeta_prop, hi) reaches alpha_floor, otherwise the bisection of
   pa_propose_schedule with alpha_target decides and theta0 sweeps are used.  Synchronising. */
pa_status pa_propose_learned(pa_ctx *ctx, const pa_learned_model *model, double alpha_floor, double alpha_target,
                             double dbeta_max, double beta_final, int theta0, int theta_max, pa_proposal *out);

/* Decorrelation of the current temperature step (a design diagnostic for the sweep count; the
   paper only asks for theta large enough to equilibrate, Sec. X): the Pearson correlation over
   replicas of the energy level right after the step's resampling and after the sweeps run so
   far at this step, from the exact integer sums of both levels, their squares and product
   (accumulated by the sweep kernel; sums_out, optional, receives them in that order).
   Synchronising. */
pa_status pa_decorrelation(pa_ctx *ctx, double *corr_out, long long *sums_out);

/* Copy up to max_entries records of the schedule run so far (one per pa_resample, in order)
   to host_out; *n_out receives the number of records available. */
pa_status pa_schedule_log(pa_ctx *ctx, pa_sched_entry *host_out, long long max_entries, long long *n_out);

/* Synchronise the stream; returns the sticky device error, if any. */
pa_status pa_sync(pa_ctx *ctx);

/* Current population size R_i (synchronising). */
pa_status pa_population(pa_ctx *ctx, long long *R_out);

/* Testing and replay accessors (all synchronising, host destinations).
   pa_histogram: N + 1 int32 level counts h_k of the current population.
   pa_replicas:  level, magnetisation and family id of replicas [0, R_i) (any may be NULL).
   pa_copy_counts: the R_{i-1} copy numbers r_j of the last resampling; host_out must hold
                 `capacity` entries, *count_out receives R_{i-1}.
   pa_hashes:    FNV-1a 64 of each replica's canonical packed bytes (rows of ceil(L/32)
                 little-endian uint32 words, bit c mod 32 of word c/32 set iff spin at
                 column c is +1).
   pa_export_spins: canonical packed words of replicas [first, first + count). */
pa_status pa_histogram(pa_ctx *ctx, int *host_out);
pa_status pa_replicas(pa_ctx *ctx, int *level, int *mag, int *fam);
pa_status pa_copy_counts(pa_ctx *ctx, int *host_out, long long *count_out);
pa_status pa_hashes(pa_ctx *ctx, unsigned long long *host_out);
pa_status pa_export_spins(pa_ctx *ctx, long long first, long long count, unsigned int *host_out);

/* ---------------------------------------------------------------------------------------
   One population split over several shards (devices or processes) by contiguous ranges of
   replica slots (Sec. II: the population is one set of R_i replicas with one normalisation
   per step, Eqs. Q and taus).  Every random number is keyed by the global slot, so the split
   does not change any result: hashes, histograms, copy numbers, family ids and observables
   are those of the same population held whole.  The caller moves data between shards; per
   temperature step each shard calls, in order:
     pa_anneal_step            theta sweeps of its own replicas and their measurement;
     pa_shard_summary          its level histogram, exact sums and family edges (device int64
                               [pa_shard_summary_len(L)]);
     (exchange)                every shard obtains all shards' summaries in slot order (an
                               all-gather);
     pa_shard_combine          the whole population's histogram, sums and family statistics,
                               identical on every shard (exact integer arithmetic);
     pa_observables/pa_record  step 4 of the whole population (optional);
     pa_resample               Eq. Q and Eq. taus from the whole histogram; copy numbers of its
                               own parents (keyed by their global index) and their offsets in
                               tree order; the children are not yet stored;
     pa_shard_layout           the number of its children c_s (synchronising);
     (exchange)                an all-gather of the c_s; their exclusive scan o_s gives the
                               children of shard s the global slots [o_s, o_s + c_s); the new
                               population is re-split into contiguous ranges of (nearly) equal
                               size [lo_t, hi_t);
     pa_shard_copy             for each range that its children meet, the children
                               [first, first + count) (local child indices) written to the given
                               arrays: the non-current buffers of the owning shard at index
                               (o_s + first - lo_t), directly when both are on one device, or a
                               staging area that the caller sends there;
     pa_shard_adopt            once every range of this shard has arrived in its non-current
                               buffers: the new local size hi_t - lo_t and slot base lo_t; the
                               non-current buffers become current.
   All three resampling kinds.  Multinomial: every shard draws all R children of the whole
   population (their random numbers are keyed by the child index) and keeps those whose draw
   falls in its parents' range of the whole population's running weight sum; the range starts
   at the weight sum of the shards before it, formed by pa_shard_combine from their
   histograms, so the copy numbers are those of the population held whole.  The
   schedule, feature, analysis and checkpoint calls need a whole population and return
   PA_ERR_STATE on a shard, as do the calls above out of order.  A shard's buffers hold its
   parents and its share of the next population, never all of its children, so its capacity
   only needs to cover its share (about R / P plus the population's fluctuation).

   pa_shard_init: cfg->R is the whole population's target size, cfg->capacity this shard's
   buffer capacity (buffers sized by pa_query_sizes for a config with R = capacity); the
   shard starts with replicas [slot_base, slot_base + R_local) of the simple-sampling
   population of step 1 (family id = global slot).  PA_ERR_INVALID_ARG unless
   0 <= slot_base, 1 <= R_local <= capacity and slot_base + R_local <= R.
   pa_shard_summary_len: int64 entries of one summary, N + 1 + 16 (0 for an unsupported L).
   pa_shard_summary: asynchronous; dev_out 8-byte aligned device memory.
   pa_shard_combine: dev_all = n_shards summaries back to back in slot order (device), one of
   them this shard's (its rows before this shard's slot base are the shards before it);
   asynchronous; an inconsistent set (histogram total != replicas, none, or no row of R_local
   replicas starting at this shard's slot base) sets the sticky error PA_ERR_NUMERIC.
   pa_shard_copy: asynchronous; spins_dst 16-byte aligned (count replicas of
   pa_sizes.bytes_per_replica bytes), level/mag/fam_dst int32[count]; children outside
   [0, c_s) are not written.
   pa_shard_adopt: asynchronous; 0 <= R_local <= capacity.
   pa_shard_layout: which buffer index (0/1) is current, the local size (after pa_resample:
   the number of children c_s) and slot base (synchronising). */
pa_status pa_shard_init(const pa_config *cfg, long long slot_base, long long R_local, const pa_buffers *buf,
                        void *stream, pa_ctx **out);
long long pa_shard_summary_len(int L);
pa_status pa_shard_summary(pa_ctx *ctx, long long *dev_out);
pa_status pa_shard_combine(pa_ctx *ctx, const long long *dev_all, int n_shards);
pa_status pa_shard_copy(pa_ctx *ctx, long long first, long long count, void *spins_dst, int *level_dst, int *mag_dst,
                        int *fam_dst);
pa_status pa_shard_adopt(pa_ctx *ctx, long long R_local, long long slot_base);
pa_status pa_shard_layout(pa_ctx *ctx, int *cur, long long *R_local, long long *slot_base);

/* Copy numbers of one resampling step WITHOUT a workspace (the paper has no counterpart: this
   is a deployment variant of the level-table / copy-number / prefix-sum kernels of
   pa_resample, not a step of the method).
   For callers that cannot provide the workspace pa_resample needs -- code that may only touch
   the arrays it is handed (e.g. a plugin inside another program's memory pool), or a process
   that fixes its device memory at start-up and forbids any later cudaMalloc.  The caller
   passes the energy levels of the R_prev parents (device int32[R_prev], level k = (E + 2N)/4)
   and receives their copy numbers r_j in counts_dev (device int32[R_prev]), exactly as
   pa_resample would draw them for the same (seed, step i, beta_prev -> beta_new, R_target,
   kind); *lnQ_out gets ln Q_i and *R_new_out the new population size.  The scratch (histogram,
   level tables, block sums) is one fixed array of 493,056 bytes in the library image, present
   on every GPU that loads the library until the process exits.  Limits: L even, 4 <= L <= 128
   (so at most 16385 levels) and 1 <= R_prev <= 4,194,304; a larger R_prev returns
   PA_ERR_TOO_LARGE.  Allocates nothing.  Every call looks up the array's device address on the
   current device (so the address stays valid across cudaDeviceReset); the first call on a
   device may also load the library's code there, so make that first call before any stream
   capture.  `stream` must belong to the current device (else PA_ERR_INVALID_ARG).  All calls
   share the array and each clears what it needs first; calls that overlap on the GPU (e.g. on
   two streams) race.  Synchronises `stream`. */
pa_status pa_copy_numbers_static(int L, long long R_target, long long R_prev, const int *level_dev,
                                 double beta_prev, double beta_new, unsigned int step,
                                 unsigned long long seed, int kind, int *counts_dev,
                                 double *lnQ_out, long long *R_new_out, void *stream);

/* ---- Batches: many independent runs of the method (Sec. II) with different L, R, number of
   temperatures, theta and seed, advanced one temperature step at a time together.  Each run
   follows the linear schedule beta_i = i / (n_temps - 1), i = 0 .. n_temps - 1 (Sec. II,
   equal steps) and computes exactly what a single-run context with the same pa_config and
   that schedule computes.  One step of every unfinished run is one replay of a captured CUDA
   graph whose sweep phase is either a single persistent launch over all runs' replicas or
   one persistent launch per lattice size (concurrent); that choice, the persistent blocks per
   SM and the replica groups per work item are chosen at initialisation by timing candidate
   shapes on the batch's own data (dry sweeps into the spare buffers, which change no run's
   state): the fastest, except that the fastest single-launch shape is kept when within 2 %
   of it. */
typedef struct pa_batch pa_batch;

typedef struct {
    pa_config cfg;     /* as for pa_init */
    int n_temps;       /* temperatures including beta_0 = 0 (>= 2) */
    int theta;         /* sweeps per temperature (>= 0) */
} pa_run_desc;

/* One shape of the batch's sweep phase tried by the autotuner. */
typedef struct {
    int unified;        /* 1: one persistent launch over every lattice size; 0: one per size,
                           concurrent on side streams */
    int blocks_per_sm;  /* persistent blocks per SM (capped by occupancy) */
    int ipw_scale;      /* replica groups per work item: the default count times this */
    float ms;           /* dry-sweep time of one step (ms) */
} pa_batch_shape;

typedef struct {
    int n_candidates;
    int chosen;                 /* index of the chosen shape */
    int chosen_grid;            /* blocks of the chosen shape's (largest) launch */
    int pad;
    pa_batch_shape cand[16];    /* the shapes tried, in order */
} pa_batch_tuning;

/* Bytes of the single caller-owned device arena (256-byte aligned) holding every run's
   buffers, workspaces and the batch tables. */
pa_status pa_batch_query_sizes(int n_runs, const pa_run_desc *runs, size_t *arena_bytes);

/* Step 1 for every run (simple sampling, measurement, records), autotuning of the sweep grid,
   and capture of the step graph.  Synchronises `stream`. */
pa_status pa_batch_init(int n_runs, const pa_run_desc *runs, void *arena, size_t arena_bytes, void *stream,
                        pa_batch **out);

/* Steps 2-4 at the next temperature of every unfinished run (finished or failed runs are
   skipped).  Asynchronous on the batch's stream. */
pa_status pa_batch_step(pa_batch *b);

/* Per run: 1 while unfinished, its pa_status, its temperature index (any may be NULL).
   Synchronising. */
pa_status pa_batch_status(pa_batch *b, int *active_out, int *status_out, long long *step_out);

/* The latest pa_obs record of every run: to device memory (asynchronous) or to the host
   (synchronising). */
pa_status pa_batch_record(pa_batch *b, void *device_dst);
pa_status pa_batch_observables(pa_batch *b, pa_obs *host_out);

/* Replica hashes of one run (as pa_hashes); host_out holds the run's capacity entries,
   *count_out receives R_i.  Synchronising. */
pa_status pa_batch_hashes(pa_batch *b, int run, unsigned long long *host_out, long long *count_out);

/* The autotuner's candidates and choice (chosen = -1 after pa_batch_set_shape). */
pa_status pa_batch_get_tuning(const pa_batch *b, pa_batch_tuning *out);

/* Replace the autotuner's choice by the given shape (ms ignored) and capture the step graph
   again; results are the same for every shape.  Synchronising; PA_ERR_INVALID_ARG for
   unified outside {0, 1}, blocks_per_sm outside [1, 32] or ipw_scale outside [1, 16]. */
pa_status pa_batch_set_shape(pa_batch *b, const pa_batch_shape *shape);

void pa_batch_destroy(pa_batch *b);

/* Checkpoint and resume (not a step of the method; the counter-based random numbers make
   the population, its exact sums, the step index, the running sum of ln Q and the schedule
   log the whole state of a run).  pa_checkpoint_size gives the bytes pa_save needs for the
   current population; pa_save writes them to host memory; pa_load restores them into a
   context created with the same pa_config, after which the run continues exactly as the
   uninterrupted one.  All synchronising; PA_ERR_INVALID_ARG for a short buffer, a foreign or
   truncated checkpoint, or a different configuration.  pa_load checks the body on the host
   before copying anything to the device and also returns PA_ERR_INVALID_ARG, leaving the
   context as it was, if the state block disagrees with the header or carries an error, or if
   an energy level lies outside [0, N], a magnetisation outside [-N, N] (or of the wrong
   parity), a family id outside [0, R) or out of tree order, or a copy number is negative or
   the copy numbers add up to more than the capacity. */
pa_status pa_checkpoint_size(pa_ctx *ctx, size_t *bytes);
pa_status pa_save(pa_ctx *ctx, void *host_buf, size_t n);
pa_status pa_load(pa_ctx *ctx, const void *host_buf, size_t n);

/* Measurement utility, not a step of the method: the rate of Philox4x32-10 alone (Salmon et
   al., SC'11, the generator of every random number above), computed as the sweep computes its
   bit planes.  Thread t of n_threads writes out_dev[t] (device uint32[n_threads], caller-owned)
   = XOR over i < calls of the four words of Philox(key = seed, ctr = (i, t, 15 << 28, 0)).
   Asynchronous on `stream` (the caller times it, e.g. with CUDA events); PA_ERR_INVALID_ARG for
   n_threads < 1, calls < 0 or a null pointer, PA_ERR_CUDA if the launch fails. */
pa_status pa_philox_xor(unsigned long long seed, int n_threads, int calls, unsigned int *out_dev, void *stream);

/* Message for the last failing call on ctx (static storage owned by the context). */
const char *pa_last_error(const pa_ctx *ctx);

/* Release the host context.  Does not touch the caller's device buffers. */
void pa_destroy(pa_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PA_H */
