// pa_api.cu -- the C ABI (include/pa.h): argument checks, the host-side context, and the
// launch sequence of each step of population annealing (arXiv:2102.06611, Sec. II).
// The library allocates no device memory; all device state lives in caller buffers.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pa_common.cuh"
#include "pa_kernels.h"

struct pa_ctx {
    pa_config cfg;
    int N;
    int device;
    int num_sms;
    cudaStream_t stream;
    pa_buffers buf;
    pa::Workspace ws;
    pa::DevState *st;
    int cur;               // index of the buffers holding the current population
    long long step;        // temperature index i
    double beta, dbeta;
    int theta_last;
    int sweeps_in_step;    // sweeps already done at this temperature
    bool measured;         // histogram and per-replica levels describe the current population
    std::vector<pa_sched_entry> log;  // one record per pa_resample
    bool prop_valid;       // the last schedule proposal, matched against the next pa_resample
    double prop_beta, prop_alpha;
    int prop_source;
    int failed;            // sticky host-side status
    char err[256];
    // one shard of a population split by contiguous slot ranges (pa_shard_*)
    bool shard;
    long long slot_base;   // global slot of local replica 0
    bool combined;         // the histogram and sums are the whole population's (pa_shard_combine)
    bool adopt_pending;    // resampled; the rebalanced population is not yet adopted
};

namespace {

bool supported_L(int L) { return L >= 4 && L <= 128 && (L % 2) == 0; }

pa_status fail(pa_ctx *c, pa_status s, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
        if (s != PA_ERR_INVALID_ARG && s != PA_ERR_STATE) c->failed = s;
    }
    return s;
}

pa_status cuda_fail(pa_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, PA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

template <typename T>
T *at(const pa_ctx *c, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(c->buf.work) + off);
}

int *cur_level(pa_ctx *c) { return static_cast<int *>(c->buf.level[c->cur]); }
int *cur_mag(pa_ctx *c) { return static_cast<int *>(c->buf.mag[c->cur]); }
int *cur_fam(pa_ctx *c) { return static_cast<int *>(c->buf.fam[c->cur]); }

// Make the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

pa_status check_live(pa_ctx *c)
{
    if (!c) return PA_ERR_INVALID_ARG;
    if (c->failed) return (pa_status)c->failed;
    return PA_OK;
}

// Calls that need the whole population in one context (schedules, features, analysis,
// checkpoints) are refused on a shard.
pa_status whole_only(pa_ctx *c, const char *what)
{
    if (c->shard) return fail(c, PA_ERR_STATE, "%s needs the whole population in one context, not a shard", what);
    return PA_OK;
}

// Synchronise and fold the device's sticky error word into the context.
pa_status sync_and_check(pa_ctx *c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    int dev_err = 0;
    e = cudaMemcpy(&dev_err, &c->st->error, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read error word");
    if (dev_err) {
        const char *what = dev_err == PA_ERR_CAPACITY ? "population exceeds buffer capacity"
                           : dev_err == PA_ERR_NUMERIC ? "empty population or non-finite weights"
                                                       : "device error";
        return fail(c, (pa_status)dev_err, "%s", what);
    }
    return PA_OK;
}

long long read_R(pa_ctx *c, bool prev, pa_status *st)
{
    long long R = 0;
    *st = sync_and_check(c);
    if (*st != PA_OK) return 0;
    cudaError_t e = cudaMemcpy(&R, prev ? &c->st->R_prev : &c->st->R_cur, sizeof(R), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) *st = cuda_fail(c, e, "read population size");
    return R;
}

// The acceptance thresholds of the sweep kernel's parameters, in the same binary64
// arithmetic as the device (pa_common.cuh: det_exp, metropolis_threshold, heatbath_threshold;
// host code is compiled without FMA contraction): Cody-Waite reduction with ln 2 split into
// a 32-bit head and a tail, degree-13 Taylor polynomial in Horner form, every operation
// rounded on its own.
double host_det_exp(double x)
{
    if (x != x) return x;
    if (x > 709.5) return HUGE_VAL;
    if (x < -745.5) return 0.0;
    const double kLn2Hi = 0x1.62e42feep-1;
    const double kLn2Lo = 0x1.a39ef35793c76p-33;
    const double kInvLn2 = 0x1.71547652b82fep+0;
    const double k = std::rint(x * kInvLn2);
    const double r = (x + -(k * kLn2Hi)) + -(k * kLn2Lo);
    const double c[14] = {1.0 / 6227020800.0, 1.0 / 479001600.0, 1.0 / 39916800.0, 1.0 / 3628800.0, 1.0 / 362880.0,
                          1.0 / 40320.0, 1.0 / 5040.0, 1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0, 1.0};
    double p = c[0];
    for (int i = 1; i < 14; ++i) p = p * r + c[i];
    return std::ldexp(p, (int)k);
}

void host_thresholds(int update, double beta, unsigned long long *T4, unsigned long long *T8)
{
    const double y4 = 4.0 * beta, y8 = 8.0 * beta;
    if (update == PA_UPDATE_HEATBATH) {
        *T4 = (unsigned long long)std::floor((1.0 / (1.0 + host_det_exp(y4))) * 4294967296.0);
        *T8 = (unsigned long long)std::floor((1.0 / (1.0 + host_det_exp(y8))) * 4294967296.0);
    } else {
        *T4 = (unsigned long long)std::floor(host_det_exp(-y4) * 4294967296.0);
        *T8 = (unsigned long long)std::floor(host_det_exp(-y8) * 4294967296.0);
    }
}

bool aligned256(const void *p) { return p && ((reinterpret_cast<uintptr_t>(p) & 255u) == 0); }

}  // namespace

extern "C" {

pa_status pa_query_sizes(const pa_config *cfg, pa_sizes *out)
{
    if (!cfg || !out) return PA_ERR_INVALID_ARG;
    if (!supported_L(cfg->L) || cfg->R < 1 || cfg->capacity < cfg->R || cfg->capacity > 2147483647LL)
        return PA_ERR_INVALID_ARG;
    if (cfg->resample != PA_RESAMPLE_NEAREST && cfg->resample != PA_RESAMPLE_POISSON &&
        cfg->resample != PA_RESAMPLE_MULTINOMIAL)
        return PA_ERR_INVALID_ARG;
    if ((cfg->update != PA_UPDATE_METROPOLIS && cfg->update != PA_UPDATE_HEATBATH) || cfg->pad != 0)
        return PA_ERR_INVALID_ARG;
    const pa::Workspace ws = pa::plan_workspace(cfg->L, cfg->capacity);
    out->bytes_per_replica = (size_t)pa::bytes_per_replica(cfg->L);
    out->spin_bytes = out->bytes_per_replica * (size_t)cfg->capacity;
    out->int_bytes = (size_t)cfg->capacity * 4;
    out->work_bytes = ws.total;
    return PA_OK;
}

}  // extern "C"

namespace {

// Context creation and step 1 (simple sampling at beta_0 = 0) for R_local replicas with
// global slots [slot_base, slot_base + R_local); a whole population has slot_base = 0 and
// R_local = cfg->R.
pa_status create_ctx(const pa_config *cfg, const pa_buffers *buf, void *stream, long long slot_base,
                     long long R_local, bool shard, pa_ctx **out)
{
    for (int b = 0; b < 2; ++b)
        if (!aligned256(buf->spins[b]) || !aligned256(buf->level[b]) || !aligned256(buf->mag[b]) ||
            !aligned256(buf->fam[b]))
            return PA_ERR_INVALID_ARG;
    if (!aligned256(buf->work)) return PA_ERR_INVALID_ARG;

    pa_ctx *c = new (std::nothrow) pa_ctx();
    if (!c) return PA_ERR_INVALID_ARG;
    c->cfg = *cfg;
    c->N = cfg->L * cfg->L;
    c->stream = static_cast<cudaStream_t>(stream);
    c->buf = *buf;
    c->ws = pa::plan_workspace(cfg->L, cfg->capacity);
    c->st = at<pa::DevState>(c, c->ws.state);
    c->cur = 0;
    c->step = 0;
    c->beta = 0.0;
    c->dbeta = 0.0;
    c->theta_last = 0;
    c->sweeps_in_step = 0;
    c->measured = true;
    c->prop_valid = false;
    c->shard = shard;
    c->slot_base = slot_base;
    c->combined = false;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return PA_ERR_CUDA;
    }
    e = pa::launch_setup(c->st, R_local, at<int>(c, c->ws.hist), c->N, cfg->update, c->stream);
    if (e == cudaSuccess) {
        pa::SweepArgs a{};
        a.spins = buf->spins[0];
        a.level = cur_level(c);
        a.mag = cur_mag(c);
        a.fam = cur_fam(c);
        a.hist = at<int>(c, c->ws.hist);
        a.st = c->st;
        a.R_init = R_local;
        a.R_bound = R_local;
        a.k0 = (unsigned int)(cfg->seed & 0xffffffffu);
        a.k1 = (unsigned int)(cfg->seed >> 32);
        a.step = 0;
        a.t0 = 0;
        a.theta = 0;
        a.slot_base = (unsigned int)slot_base;
        host_thresholds(cfg->update, 0.0, &a.T4, &a.T8);
        e = pa::launch_sweep(cfg->L, true, a, c->num_sms, c->stream);
    }
    if (e != cudaSuccess) {
        delete c;
        return PA_ERR_CUDA;
    }
    *out = c;
    return PA_OK;
}

}  // namespace

extern "C" {

pa_status pa_init(const pa_config *cfg, const pa_buffers *buf, void *stream, pa_ctx **out)
{
    if (!out) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    pa_sizes sz;
    if (!cfg || !buf || pa_query_sizes(cfg, &sz) != PA_OK) return PA_ERR_INVALID_ARG;
    return create_ctx(cfg, buf, stream, 0, cfg->R, false, out);
}

pa_status pa_shard_init(const pa_config *cfg, long long slot_base, long long R_local, const pa_buffers *buf,
                        void *stream, pa_ctx **out)
{
    if (!out) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || !buf) return PA_ERR_INVALID_ARG;
    // the buffers hold `capacity` replicas of this shard; cfg->R is the whole population's target
    pa_config local = *cfg;
    local.R = local.capacity;
    pa_sizes sz;
    if (pa_query_sizes(&local, &sz) != PA_OK || cfg->R < 1 || cfg->R > 2147483647LL) return PA_ERR_INVALID_ARG;
    if (slot_base < 0 || R_local < 1 || R_local > cfg->capacity || slot_base + R_local > cfg->R)
        return PA_ERR_INVALID_ARG;
    return create_ctx(cfg, buf, stream, slot_base, R_local, true, out);
}

static pa_status sweep_and_measure(pa_ctx *c, int theta);

pa_status pa_resample(pa_ctx *c, double beta_new)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!std::isfinite(beta_new) || beta_new < c->beta)
        return fail(c, PA_ERR_STATE, "beta_new %.17g must be finite and >= current beta %.17g", beta_new, c->beta);
    if (c->shard && (!c->combined || c->adopt_pending))
        return fail(c, PA_ERR_STATE, "a shard resamples after pa_shard_combine of the current measurement");
    DeviceGuard g(c->device);
    // Eqs. Q and taus need the parents' histogram: measure a population resampled again
    // without a sweep in between (a shard's histogram is the combined one)
    if (!c->shard && !c->measured && (s = sweep_and_measure(c, 0)) != PA_OK) return s;
    const int nxt = c->cur ^ 1;
    pa::ResampleArgs a{};
    a.sharded = c->shard ? 1 : 0;
    a.parent_base = (unsigned int)c->slot_base;
    a.hist_before = at<int>(c, c->ws.hist_before);
    a.L = c->cfg.L;
    a.kind = c->cfg.resample;
    a.R_target = c->cfg.R;
    a.capacity = c->cfg.capacity;
    a.beta_prev = c->beta;
    a.beta_new = beta_new;
    a.step = (unsigned int)(c->step + 1);
    a.k0 = (unsigned int)(c->cfg.seed & 0xffffffffu);
    a.k1 = (unsigned int)(c->cfg.seed >> 32);
    a.st = c->st;
    a.hist = at<int>(c, c->ws.hist);
    a.fl = at<int>(c, c->ws.fl);
    a.thr = at<unsigned int>(c, c->ws.thr);
    a.tau = at<double>(c, c->ws.tau);
    a.w = at<double>(c, c->ws.w);
    a.counts = at<int>(c, c->ws.counts);
    a.blocksum = at<long long>(c, c->ws.blocksum);
    a.nblk = c->ws.nblk;
    a.wint = at<unsigned long long>(c, c->ws.wint);
    a.cdf = at<unsigned long long>(c, c->ws.cdf);
    a.spins_src = c->buf.spins[c->cur];
    a.spins_dst = c->buf.spins[nxt];
    a.level_src = static_cast<const int *>(c->buf.level[c->cur]);
    a.mag_src = static_cast<const int *>(c->buf.mag[c->cur]);
    a.fam_src = static_cast<const int *>(c->buf.fam[c->cur]);
    a.level_dst = static_cast<int *>(c->buf.level[nxt]);
    a.mag_dst = static_cast<int *>(c->buf.mag[nxt]);
    a.fam_dst = static_cast<int *>(c->buf.fam[nxt]);
    // a shard only draws its parents' copy numbers here: its children are copied by
    // pa_shard_copy into the shards that own their global slots
    cudaError_t e = c->shard ? pa::launch_copy_numbers(a, c->stream) : pa::launch_resample(a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "resample launch");
    if (!c->shard) c->cur = nxt;
    c->step += 1;
    c->dbeta = beta_new - c->beta;
    pa_sched_entry rec{};
    rec.step = c->step;
    rec.beta = beta_new;
    rec.dbeta = c->dbeta;
    rec.theta = 0;
    const bool proposed = c->prop_valid && beta_new == c->prop_beta;
    rec.source = proposed ? c->prop_source : PA_SCHED_CALLER;
    rec.alpha = proposed ? c->prop_alpha : std::nan("");
    c->log.push_back(rec);
    c->prop_valid = false;
    c->beta = beta_new;
    c->sweeps_in_step = 0;
    c->measured = false;
    c->combined = false;
    c->adopt_pending = c->shard;
    return PA_OK;
}

// theta sweeps at the current beta (theta = 0: measurement only), then energies, magnetisations
// and the level histogram of the current population.
static pa_status sweep_and_measure(pa_ctx *c, int theta)
{
    cudaError_t e = pa::launch_zero_measure(c->st, at<int>(c, c->ws.hist), c->N, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "zero measurement");
    pa::SweepArgs a{};
    a.spins = c->buf.spins[c->cur];
    a.level = cur_level(c);
    a.mag = cur_mag(c);
    a.fam = cur_fam(c);
    a.level_snap = at<int>(c, c->ws.snap);
    a.hist = at<int>(c, c->ws.hist);
    a.st = c->st;
    a.R_init = 0;
    a.R_bound = c->cfg.capacity;
    a.k0 = (unsigned int)(c->cfg.seed & 0xffffffffu);
    a.k1 = (unsigned int)(c->cfg.seed >> 32);
    a.step = (unsigned int)c->step;
    a.t0 = c->sweeps_in_step;
    a.theta = theta;
    a.update = c->cfg.update;
    a.slot_base = (unsigned int)c->slot_base;
    host_thresholds(c->cfg.update, c->beta, &a.T4, &a.T8);
    e = pa::launch_sweep(c->cfg.L, false, a, c->num_sms, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep launch");
    c->measured = true;
    c->combined = false;
    return PA_OK;
}

pa_status pa_anneal_step(pa_ctx *c, int theta)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (theta < 0 || (long long)c->sweeps_in_step + theta > (1 << 27))
        return fail(c, PA_ERR_INVALID_ARG, "theta %d out of range", theta);
    if (c->adopt_pending) return fail(c, PA_ERR_STATE, "a shard adopts its rebalanced population before sweeping");
    DeviceGuard g(c->device);
    if ((s = sweep_and_measure(c, theta)) != PA_OK) return s;
    c->sweeps_in_step += theta;
    c->theta_last = theta;
    if (!c->log.empty() && c->log.back().step == c->step) c->log.back().theta += theta;
    return PA_OK;
}

pa_status pa_propose_schedule(pa_ctx *c, double alpha_target, double dbeta_max, double beta_final,
                              double *beta_next, double *alpha_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "the adaptive schedule")) != PA_OK) return s;
    if (!beta_next || !alpha_out || !(alpha_target > 0.0 && alpha_target <= 1.0) || !(dbeta_max > 0.0) ||
        !std::isfinite(dbeta_max) || !std::isfinite(beta_final))
        return fail(c, PA_ERR_INVALID_ARG, "bad schedule parameters");
    if (beta_final < c->beta)
        return fail(c, PA_ERR_STATE, "beta_final %.17g below current beta %.17g", beta_final, c->beta);
    DeviceGuard g(c->device);
    if (!c->measured && (s = sweep_and_measure(c, 0)) != PA_OK) return s;
    pa::BisectArgs a{};
    a.L = c->cfg.L;
    a.st = c->st;
    a.hist = at<int>(c, c->ws.hist);
    a.occ_k = at<int>(c, c->ws.occ_k);
    a.occ_h = at<int>(c, c->ws.occ_h);
    a.occ_w = at<double>(c, c->ws.occ_w);
    a.occ_t = at<double>(c, c->ws.occ_t);
    a.beta = c->beta;
    a.beta_final = beta_final;
    a.dbeta_max = dbeta_max;
    a.alpha_target = alpha_target;
    a.iters = pa::kBisectIters;
    cudaError_t e = pa::launch_bisect(a, at<pa::SearchState>(c, c->ws.search), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "bisection launch");
    if ((s = sync_and_check(c)) != PA_OK) return s;
    double out[2];
    e = cudaMemcpy(out, &c->st->beta_next, sizeof(out), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "proposal copy");
    *beta_next = out[0];
    *alpha_out = out[1];
    c->prop_valid = true;
    c->prop_beta = out[0];
    c->prop_alpha = out[1];
    c->prop_source = PA_SCHED_BISECT;
    return PA_OK;
}

pa_status pa_decorrelation(pa_ctx *c, double *corr_out, long long *sums_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "the decorrelation measure")) != PA_OK) return s;
    if (!corr_out) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!c->measured && (s = sweep_and_measure(c, 0)) != PA_OK) return s;
    if ((s = sync_and_check(c)) != PA_OK) return s;
    long long v[5];
    long long R;
    cudaError_t e = cudaMemcpy(v, &c->st->c0, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&R, &c->st->R_cur, sizeof(R), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "correlation sums copy");
    // corr = cov(k0, k1) / sqrt(var k0 var k1), all from exact integer sums
    const double Rd = (double)R;
    const double cov = (double)v[4] - (double)v[0] * (double)v[2] / Rd;
    const double v0 = (double)v[1] - (double)v[0] * (double)v[0] / Rd;
    const double v1 = (double)v[3] - (double)v[2] * (double)v[2] / Rd;
    *corr_out = (v0 > 0.0 && v1 > 0.0) ? cov / std::sqrt(v0 * v1) : 0.0;
    if (sums_out)
        for (int i = 0; i < 5; ++i) sums_out[i] = v[i];
    return PA_OK;
}

// Features of the current population on the device (raw in feat[0..11], standardised in
// feat[16..27]); the previous-step inputs come from the schedule log.
static pa_status launch_feature_pass(pa_ctx *c, int theta0, const float *norm)
{
    pa_status s;
    if (!c->measured && (s = sweep_and_measure(c, 0)) != PA_OK) return s;
    cudaError_t e = pa::launch_families(c->st, cur_fam(c), at<long long>(c, c->ws.fampart), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "families launch");
    pa::FeatureArgs a{};
    a.L = c->cfg.L;
    a.st = c->st;
    a.hist = at<int>(c, c->ws.hist);
    a.fampart = at<long long>(c, c->ws.fampart);
    a.counts = at<int>(c, c->ws.counts);
    a.beta = c->beta;
    a.dbeta_prev = c->dbeta;
    const bool have = !c->log.empty();
    a.theta_ratio_prev = have ? (double)c->log.back().theta / (double)theta0 : 0.0;
    a.alpha_prev = (have && std::isfinite(c->log.back().alpha)) ? c->log.back().alpha : 1.0;
    a.norm = norm;
    a.raw = at<float>(c, c->ws.feat);
    a.x = at<float>(c, c->ws.feat) + 16;
    a.zeros = reinterpret_cast<unsigned long long *>(at<float>(c, c->ws.feat) + 32);
    a.capacity = c->cfg.capacity;
    e = pa::launch_features(a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "features launch");
    return PA_OK;
}

pa_status pa_features(pa_ctx *c, int theta0, float *host_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "the schedule features")) != PA_OK) return s;
    if (!host_out || theta0 < 1) return fail(c, PA_ERR_INVALID_ARG, "bad feature arguments");
    DeviceGuard g(c->device);
    if ((s = launch_feature_pass(c, theta0, nullptr)) != PA_OK) return s;
    if ((s = sync_and_check(c)) != PA_OK) return s;
    cudaError_t e = cudaMemcpy(host_out, at<float>(c, c->ws.feat), 12 * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "feature copy");
}

pa_status pa_propose_learned(pa_ctx *c, const pa_learned_model *model, double alpha_floor, double alpha_target,
                             double dbeta_max, double beta_final, int theta0, int theta_max, pa_proposal *out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "the learned schedule")) != PA_OK) return s;
    if (!model || !model->params_bf16 || !model->norm || !out || theta0 < 1 || theta_max < 1 ||
        !(alpha_floor > 0.0 && alpha_floor <= 1.0) || !(alpha_target > 0.0 && alpha_target <= 1.0) ||
        !(dbeta_max > 0.0) || !std::isfinite(dbeta_max) || !std::isfinite(beta_final))
        return fail(c, PA_ERR_INVALID_ARG, "bad learned-schedule arguments");
    if (beta_final < c->beta)
        return fail(c, PA_ERR_STATE, "beta_final %.17g below current beta %.17g", beta_final, c->beta);
    DeviceGuard g(c->device);
    if ((s = launch_feature_pass(c, theta0, model->norm)) != PA_OK) return s;
    cudaError_t e = pa::launch_mlp_propose(model->params_bf16, model->norm, at<float>(c, c->ws.feat),
                                           at<float>(c, c->ws.feat) + 16,
                                           c->cfg.L, dbeta_max, theta_max, c->st, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "network launch");
    pa::BisectArgs a{};
    a.L = c->cfg.L;
    a.st = c->st;
    a.hist = at<int>(c, c->ws.hist);
    a.occ_k = at<int>(c, c->ws.occ_k);
    a.occ_h = at<int>(c, c->ws.occ_h);
    a.occ_w = at<double>(c, c->ws.occ_w);
    a.occ_t = at<double>(c, c->ws.occ_t);
    a.beta = c->beta;
    a.beta_final = beta_final;
    a.dbeta_max = dbeta_max;
    a.alpha_target = alpha_target;
    a.iters = pa::kBisectIters;
    a.use_prop = 1;
    a.alpha_floor = alpha_floor;
    e = pa::launch_bisect(a, at<pa::SearchState>(c, c->ws.search), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "proposal check launch");
    if ((s = sync_and_check(c)) != PA_OK) return s;
    pa::DevState h;
    e = cudaMemcpy(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "proposal copy");
    out->beta_next = h.beta_next;
    out->alpha = h.alpha_next;
    out->dbeta_prop = h.dbeta_prop;
    out->theta_prop = h.theta_prop;
    out->source = h.source_next;
    out->theta_next = h.source_next == PA_SCHED_LEARNED ? h.theta_prop : theta0;
    out->pad = 0;
    c->prop_valid = true;
    c->prop_beta = h.beta_next;
    c->prop_alpha = h.alpha_next;
    c->prop_source = h.source_next;
    return PA_OK;
}

pa_status pa_schedule_log(pa_ctx *c, pa_sched_entry *host_out, long long max_entries, long long *n_out)
{
    if (!c || !n_out || max_entries < 0 || (max_entries > 0 && !host_out)) return PA_ERR_INVALID_ARG;
    const long long n = (long long)c->log.size();
    *n_out = n;
    for (long long i = 0; i < n && i < max_entries; ++i) host_out[i] = c->log[(size_t)i];
    return PA_OK;
}

pa_status pa_record(pa_ctx *c, void *device_dst)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!device_dst || (reinterpret_cast<uintptr_t>(device_dst) & 7u))
        return fail(c, PA_ERR_INVALID_ARG, "record destination must be an 8-byte aligned device pointer");
    if (c->shard && !(c->measured && c->combined))
        return fail(c, PA_ERR_STATE, "a shard reports observables after pa_shard_combine of its measurement");
    DeviceGuard g(c->device);
    if (!c->measured && (s = sweep_and_measure(c, 0)) != PA_OK) return s;
    pa::ObsArgs a{};
    a.glob = c->shard ? 1 : 0;
    a.L = c->cfg.L;
    a.R_target = c->cfg.R;
    a.step = c->step;
    a.beta = c->beta;
    a.dbeta = c->dbeta;
    a.theta = c->theta_last;
    a.st = c->st;
    a.hist = at<int>(c, c->ws.hist);
    a.fam = cur_fam(c);
    a.fampart = at<long long>(c, c->ws.fampart);
    a.dst = static_cast<pa_obs *>(device_dst);
    cudaError_t e = pa::launch_observables(a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "observables launch");
    return PA_OK;
}

pa_status pa_observables(pa_ctx *c, pa_obs *host_out)
{
    if (!host_out) return PA_ERR_INVALID_ARG;
    pa_status s = pa_record(c, at<void>(c, c->ws.obs));
    if (s != PA_OK) return s;
    DeviceGuard g(c->device);
    cudaError_t e = cudaMemcpyAsync(host_out, at<void>(c, c->ws.obs), sizeof(pa_obs), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "observables copy");
    return sync_and_check(c);
}

pa_status pa_weighted_average(const void *records_dev, int M, int mode, void *out_dev, void *stream)
{
    if (!records_dev || !out_dev || M < 1 || (mode != 0 && mode != 1) ||
        (reinterpret_cast<uintptr_t>(records_dev) & 7u) || (reinterpret_cast<uintptr_t>(out_dev) & 7u))
        return PA_ERR_INVALID_ARG;
    cudaError_t e = pa::launch_weighted(static_cast<const pa_obs *>(records_dev), M, mode,
                                        static_cast<pa_weighted *>(out_dev), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_analyze(pa_ctx *c, int n_blocks, pa_analysis *host_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "the population analysis")) != PA_OK) return s;
    if (!host_out || n_blocks < 2 || n_blocks > pa::kMaxAnaBlocks)
        return fail(c, PA_ERR_INVALID_ARG, "n_blocks %d outside [2, %d]", n_blocks, pa::kMaxAnaBlocks);
    DeviceGuard g(c->device);
    if (!c->measured && (s = sweep_and_measure(c, 0)) != PA_OK) return s;
    const long long R = read_R(c, false, &s);
    if (s != PA_OK) return s;
    if ((long long)n_blocks > R) return fail(c, PA_ERR_INVALID_ARG, "n_blocks %d above R_i = %lld", n_blocks, R);
    cudaError_t e = pa::launch_analysis(c->st, cur_level(c), cur_mag(c), cur_fam(c), c->N, c->beta, n_blocks,
                                        c->cfg.capacity, at<long long>(c, c->ws.ana_blk), at<int>(c, c->ws.ana_sizes),
                                        at<pa_analysis>(c, c->ws.ana_out), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "analysis launch");
    e = cudaMemcpyAsync(host_out, at<void>(c, c->ws.ana_out), sizeof(pa_analysis), cudaMemcpyDeviceToHost,
                        c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "analysis copy");
    return sync_and_check(c);
}

pa_status pa_sync(pa_ctx *c)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    DeviceGuard g(c->device);
    return sync_and_check(c);
}

pa_status pa_population(pa_ctx *c, long long *R_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!R_out) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    *R_out = read_R(c, false, &s);
    return s;
}

pa_status pa_histogram(pa_ctx *c, int *host_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!host_out) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if ((s = sync_and_check(c)) != PA_OK) return s;
    cudaError_t e = cudaMemcpy(host_out, at<int>(c, c->ws.hist), sizeof(int) * (size_t)(c->N + 1),
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "histogram copy");
}

pa_status pa_replicas(pa_ctx *c, int *level, int *mag, int *fam)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (c->adopt_pending) return fail(c, PA_ERR_STATE, "the shard's children are not adopted yet");
    DeviceGuard g(c->device);
    const long long R = read_R(c, false, &s);
    if (s != PA_OK) return s;
    const size_t bytes = sizeof(int) * (size_t)R;
    cudaError_t e = cudaSuccess;
    if (level && e == cudaSuccess) e = cudaMemcpy(level, cur_level(c), bytes, cudaMemcpyDeviceToHost);
    if (mag && e == cudaSuccess) e = cudaMemcpy(mag, cur_mag(c), bytes, cudaMemcpyDeviceToHost);
    if (fam && e == cudaSuccess) e = cudaMemcpy(fam, cur_fam(c), bytes, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "replica copy");
}

pa_status pa_copy_counts(pa_ctx *c, int *host_out, long long *count_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!host_out || !count_out) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    const long long Rp = read_R(c, true, &s);
    if (s != PA_OK) return s;
    *count_out = Rp;
    cudaError_t e = cudaMemcpy(host_out, at<int>(c, c->ws.counts), sizeof(int) * (size_t)Rp,
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "copy-count copy");
}

pa_status pa_hashes(pa_ctx *c, unsigned long long *host_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (c->adopt_pending) return fail(c, PA_ERR_STATE, "the shard's children are not adopted yet");
    if (!host_out) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    unsigned long long *dev = at<unsigned long long>(c, c->ws.hashes);
    cudaError_t e = pa::launch_hashes(c->cfg.L, c->buf.spins[c->cur], c->cfg.capacity, c->st, dev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "hash launch");
    const long long R = read_R(c, false, &s);
    if (s != PA_OK) return s;
    e = cudaMemcpy(host_out, dev, sizeof(unsigned long long) * (size_t)R, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "hash copy");
}

pa_status pa_export_spins(pa_ctx *c, long long first, long long count, unsigned int *host_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (c->adopt_pending) return fail(c, PA_ERR_STATE, "the shard's children are not adopted yet");
    if (!host_out || first < 0 || count < 0) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    const long long R = read_R(c, false, &s);
    if (s != PA_OK) return s;
    if (first + count > R) return fail(c, PA_ERR_INVALID_ARG, "replicas [%lld, %lld) beyond R = %lld", first,
                                       first + count, R);
    const size_t words = (size_t)c->cfg.L * ((c->cfg.L + 31) / 32);
    unsigned int *stage = at<unsigned int>(c, c->ws.stage);
    for (long long done = 0; done < count; done += pa::kStageReplicas) {
        const long long n = count - done < pa::kStageReplicas ? count - done : pa::kStageReplicas;
        cudaError_t e = pa::launch_export(c->cfg.L, c->buf.spins[c->cur], first + done, n, stage, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_out + (size_t)done * words, stage, sizeof(unsigned int) * words * (size_t)n,
                                cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "spin export");
    }
    return PA_OK;
}

// ------------------------------------------------------------------------------ checkpoints
// Layout: header, device state block, level histogram, then per replica of the current
// population the packed spins, level, magnetisation, family id and step-start level, then the
// R_{i-1} copy numbers of the last resampling, then the schedule log.  The random numbers are
// counter based, so this is the whole state of a run.
namespace {
constexpr unsigned long long kCkptMagic = 0x3131363630323150ull;  // "P2066611" tag
struct CkptHeader {
    unsigned long long magic;
    pa_config cfg;
    long long step, R_cur, R_prev, n_log;
    double beta, dbeta;
    int sweeps_in_step, theta_last, measured, version;
};

size_t ckpt_bytes(const pa_ctx *c, long long R, long long Rp, long long nlog)
{
    const size_t bpr = (size_t)pa::bytes_per_replica(c->cfg.L);
    return sizeof(CkptHeader) + sizeof(pa::DevState) + sizeof(int) * (size_t)(c->N + 1) +
           (size_t)R * (bpr + 4 * sizeof(int)) + (size_t)Rp * sizeof(int) + (size_t)nlog * sizeof(pa_sched_entry);
}

// Host-side check of a checkpoint body before anything reaches the device: the kernels bound
// their loops by the state block's R_cur / R_prev and index the level tables by stored energy
// levels, so a file whose state block disagrees with its header, or whose levels, family ids,
// magnetisations or copy numbers are out of range, is rejected here instead of driving
// out-of-range device accesses.  Returns null if the body is consistent, else the reason.
const char *ckpt_invalid(const pa_ctx *c, const CkptHeader &h, const char *p)
{
    const int N = c->N;
    if (h.step < 0 || h.sweeps_in_step < 0 || h.theta_last < 0 || (h.measured != 0 && h.measured != 1) ||
        !std::isfinite(h.beta) || !std::isfinite(h.dbeta))
        return "header fields out of range";
    pa::DevState ds;
    std::memcpy(&ds, p, sizeof(ds));
    p += sizeof(ds);
    if (ds.R_cur != h.R_cur || ds.R_prev != h.R_prev) return "state block sizes differ from the header";
    if (ds.error != 0) return "state block carries an error";
    if (ds.update != c->cfg.update || ds.kmin < 0 || ds.kmin > N || ds.theta < 0 ||
        ds.T4 > (1ull << 32) || ds.T8 > (1ull << 32))
        return "state block fields out of range";
    auto ints = [&p](long long n) {
        const char *q = p;
        p += sizeof(int) * (size_t)n;
        return q;
    };
    auto get = [](const char *base, long long j) {
        int v;
        std::memcpy(&v, base + sizeof(int) * (size_t)j, sizeof(v));
        return v;
    };
    const char *hist = ints(N + 1);
    for (int k = 0; k <= N; ++k)
        if (get(hist, k) < 0) return "negative histogram entry";
    p += (size_t)pa::bytes_per_replica(c->cfg.L) * (size_t)h.R_cur;
    const char *level = ints(h.R_cur), *mag = ints(h.R_cur), *fam = ints(h.R_cur), *snap = ints(h.R_cur);
    const char *counts = ints(h.R_prev);
    for (long long j = 0; j < h.R_cur; ++j) {
        const int k = get(level, j), m = get(mag, j), f = get(fam, j), k0 = get(snap, j);
        // the step-start levels are written by the step's first sweep and read only after it
        if (k < 0 || k > N || (h.sweeps_in_step > 0 && (k0 < 0 || k0 > N))) return "energy level out of range";
        if (m < -N || m > N || ((m + N) & 1)) return "magnetisation out of range";
        if (f < 0 || f >= c->cfg.R || (j > 0 && f < get(fam, j - 1))) return "family ids out of range or order";
    }
    long long total = 0;
    for (long long j = 0; j < h.R_prev; ++j) {
        const int r = get(counts, j);
        if (r < 0) return "negative copy number";
        total += r;
    }
    if (total > c->cfg.capacity) return "copy numbers exceed the capacity";
    return nullptr;
}

pa_status read_sizes(pa_ctx *c, long long *R, long long *Rp)
{
    pa_status s = sync_and_check(c);
    if (s != PA_OK) return s;
    cudaError_t e = cudaMemcpy(R, &c->st->R_cur, sizeof(*R), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(Rp, &c->st->R_prev, sizeof(*Rp), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "checkpoint sizes");
}
}  // namespace

pa_status pa_checkpoint_size(pa_ctx *c, size_t *bytes)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "a checkpoint")) != PA_OK) return s;
    if (!bytes) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    long long R, Rp;
    if ((s = read_sizes(c, &R, &Rp)) != PA_OK) return s;
    *bytes = ckpt_bytes(c, R, Rp, (long long)c->log.size());
    return PA_OK;
}

pa_status pa_save(pa_ctx *c, void *host_buf, size_t n)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "a checkpoint")) != PA_OK) return s;
    if (!host_buf) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    long long R, Rp;
    if ((s = read_sizes(c, &R, &Rp)) != PA_OK) return s;
    if (n < ckpt_bytes(c, R, Rp, (long long)c->log.size()))
        return fail(c, PA_ERR_INVALID_ARG, "checkpoint buffer of %zu bytes is too small", n);
    char *p = static_cast<char *>(host_buf);
    CkptHeader h{};
    h.magic = kCkptMagic;
    h.version = 3;
    h.cfg = c->cfg;
    h.step = c->step;
    h.R_cur = R;
    h.R_prev = Rp;
    h.n_log = (long long)c->log.size();
    h.beta = c->beta;
    h.dbeta = c->dbeta;
    h.sweeps_in_step = c->sweeps_in_step;
    h.theta_last = c->theta_last;
    h.measured = c->measured ? 1 : 0;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t bpr = (size_t)pa::bytes_per_replica(c->cfg.L);
    struct Piece { const void *src; size_t bytes; } pieces[] = {
        {c->st, sizeof(pa::DevState)},
        {at<int>(c, c->ws.hist), sizeof(int) * (size_t)(c->N + 1)},
        {c->buf.spins[c->cur], bpr * (size_t)R},
        {c->buf.level[c->cur], sizeof(int) * (size_t)R},
        {c->buf.mag[c->cur], sizeof(int) * (size_t)R},
        {c->buf.fam[c->cur], sizeof(int) * (size_t)R},
        {at<int>(c, c->ws.snap), sizeof(int) * (size_t)R},
        {at<int>(c, c->ws.counts), sizeof(int) * (size_t)Rp},
    };
    for (const Piece &q : pieces) {
        cudaError_t e = cudaMemcpy(p, q.src, q.bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
        p += q.bytes;
    }
    if (!c->log.empty()) std::memcpy(p, c->log.data(), sizeof(pa_sched_entry) * c->log.size());
    return PA_OK;
}

pa_status pa_load(pa_ctx *c, const void *host_buf, size_t n)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if ((s = whole_only(c, "a checkpoint")) != PA_OK) return s;
    if (!host_buf || n < sizeof(CkptHeader)) return PA_ERR_INVALID_ARG;
    CkptHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (h.magic != kCkptMagic || h.version != 3) return fail(c, PA_ERR_INVALID_ARG, "not a checkpoint");
    if (std::memcmp(&h.cfg, &c->cfg, sizeof(pa_config)) != 0)
        return fail(c, PA_ERR_INVALID_ARG, "checkpoint of a different configuration");
    if (h.R_cur < 1 || h.R_cur > c->cfg.capacity || h.R_prev < 0 || h.R_prev > c->cfg.capacity || h.n_log < 0 ||
        n < ckpt_bytes(c, h.R_cur, h.R_prev, h.n_log))
        return fail(c, PA_ERR_INVALID_ARG, "truncated or inconsistent checkpoint");
    if (const char *why = ckpt_invalid(c, h, static_cast<const char *>(host_buf) + sizeof(h)))
        return fail(c, PA_ERR_INVALID_ARG, "invalid checkpoint: %s", why);
    DeviceGuard g(c->device);
    if ((s = sync_and_check(c)) != PA_OK) return s;
    const char *p = static_cast<const char *>(host_buf) + sizeof(h);
    c->cur = 0;
    const size_t bpr = (size_t)pa::bytes_per_replica(c->cfg.L);
    struct Piece { void *dst; size_t bytes; } pieces[] = {
        {c->st, sizeof(pa::DevState)},
        {at<int>(c, c->ws.hist), sizeof(int) * (size_t)(c->N + 1)},
        {c->buf.spins[0], bpr * (size_t)h.R_cur},
        {c->buf.level[0], sizeof(int) * (size_t)h.R_cur},
        {c->buf.mag[0], sizeof(int) * (size_t)h.R_cur},
        {c->buf.fam[0], sizeof(int) * (size_t)h.R_cur},
        {at<int>(c, c->ws.snap), sizeof(int) * (size_t)h.R_cur},
        {at<int>(c, c->ws.counts), sizeof(int) * (size_t)h.R_prev},
    };
    for (const Piece &q : pieces) {
        cudaError_t e = cudaMemcpy(q.dst, p, q.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint restore");
        p += q.bytes;
    }
    c->log.assign(reinterpret_cast<const pa_sched_entry *>(p), reinterpret_cast<const pa_sched_entry *>(p) + h.n_log);
    c->step = h.step;
    c->beta = h.beta;
    c->dbeta = h.dbeta;
    c->sweeps_in_step = h.sweeps_in_step;
    c->theta_last = h.theta_last;
    c->measured = h.measured != 0;
    c->prop_valid = false;
    return PA_OK;
}

// ------------------------------------------------------------------------------ shards
long long pa_shard_summary_len(int L)
{
    if (!supported_L(L)) return 0;
    return (long long)L * L + 1 + pa::kShardExtra;
}

pa_status pa_shard_summary(pa_ctx *c, long long *dev_out)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!c->shard) return fail(c, PA_ERR_STATE, "pa_shard_summary needs a shard context");
    if (!dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 7u))
        return fail(c, PA_ERR_INVALID_ARG, "summary destination must be an 8-byte aligned device pointer");
    if (c->combined || c->adopt_pending)
        return fail(c, PA_ERR_STATE, "summarise a shard once after each measurement");
    DeviceGuard g(c->device);
    if (!c->measured && (s = sweep_and_measure(c, 0)) != PA_OK) return s;
    cudaError_t e = pa::launch_families(c->st, cur_fam(c), at<long long>(c, c->ws.fampart), c->stream);
    if (e == cudaSuccess)
        e = pa::launch_shard_summary(c->st, at<int>(c, c->ws.hist), cur_fam(c), at<long long>(c, c->ws.fampart), c->N,
                                     dev_out, c->stream);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "shard summary launch");
}

pa_status pa_shard_combine(pa_ctx *c, const long long *dev_all, int n_shards)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!c->shard) return fail(c, PA_ERR_STATE, "pa_shard_combine needs a shard context");
    if (!dev_all || n_shards < 1 || (reinterpret_cast<uintptr_t>(dev_all) & 7u))
        return fail(c, PA_ERR_INVALID_ARG, "bad shard summaries");
    if (!c->measured || c->combined) return fail(c, PA_ERR_STATE, "combine once after each measurement");
    DeviceGuard g(c->device);
    cudaError_t e = pa::launch_shard_combine(c->st, at<int>(c, c->ws.hist), at<int>(c, c->ws.hist_before), c->slot_base,
                                             c->N, dev_all, n_shards, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "shard combine launch");
    c->combined = true;
    return PA_OK;
}

pa_status pa_shard_copy(pa_ctx *c, long long first, long long count, void *spins_dst, int *level_dst, int *mag_dst,
                        int *fam_dst)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!c->shard) return fail(c, PA_ERR_STATE, "pa_shard_copy needs a shard context");
    if (!c->adopt_pending) return fail(c, PA_ERR_STATE, "pa_shard_copy follows pa_resample");
    if (first < 0 || count < 0 || !spins_dst || !level_dst || !mag_dst || !fam_dst ||
        (reinterpret_cast<uintptr_t>(spins_dst) & 15u) || (reinterpret_cast<uintptr_t>(level_dst) & 3u) ||
        (reinterpret_cast<uintptr_t>(mag_dst) & 3u) || (reinterpret_cast<uintptr_t>(fam_dst) & 3u))
        return fail(c, PA_ERR_INVALID_ARG, "bad children window or destination");
    if (count == 0) return PA_OK;
    DeviceGuard g(c->device);
    pa::ResampleArgs a{};
    a.L = c->cfg.L;
    a.st = c->st;
    a.counts = at<int>(c, c->ws.counts);
    a.blocksum = at<long long>(c, c->ws.blocksum);
    a.nblk = c->ws.nblk;
    a.spins_src = c->buf.spins[c->cur];
    a.level_src = static_cast<const int *>(c->buf.level[c->cur]);
    a.mag_src = static_cast<const int *>(c->buf.mag[c->cur]);
    a.fam_src = static_cast<const int *>(c->buf.fam[c->cur]);
    a.spins_dst = spins_dst;
    a.level_dst = level_dst;
    a.mag_dst = mag_dst;
    a.fam_dst = fam_dst;
    a.sharded = 1;
    a.win_lo = first;
    a.win_n = count;
    cudaError_t e = pa::launch_copy(a, c->stream);
    return e == cudaSuccess ? PA_OK : cuda_fail(c, e, "shard copy launch");
}

pa_status pa_shard_adopt(pa_ctx *c, long long R_local, long long slot_base)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!c->shard) return fail(c, PA_ERR_STATE, "pa_shard_adopt needs a shard context");
    if (!c->adopt_pending) return fail(c, PA_ERR_STATE, "pa_shard_adopt follows pa_resample");
    if (R_local < 0 || R_local > c->cfg.capacity || slot_base < 0 || slot_base + R_local > 2147483647LL)
        return fail(c, PA_ERR_INVALID_ARG, "R_local %lld / slot_base %lld out of range", R_local, slot_base);
    DeviceGuard g(c->device);
    cudaError_t e = pa::launch_set_population(c->st, R_local, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "shard adopt launch");
    c->cur ^= 1;
    c->slot_base = slot_base;
    c->adopt_pending = false;
    return PA_OK;
}

pa_status pa_shard_layout(pa_ctx *c, int *cur, long long *R_local, long long *slot_base)
{
    pa_status s = check_live(c);
    if (s != PA_OK) return s;
    if (!cur || !R_local || !slot_base) return PA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    const long long R = read_R(c, false, &s);
    if (s != PA_OK) return s;
    *cur = c->cur;
    *R_local = R;
    *slot_base = c->slot_base;
    return PA_OK;
}

const char *pa_last_error(const pa_ctx *c)
{
    if (!c) return "null context";
    return c->err;
}

void pa_destroy(pa_ctx *c)
{
    delete c;
}

}  // extern "C"
