// pa_batch.cu -- many independent population-annealing runs (different L, R, number of
// temperatures, theta, seed) advanced together: one captured CUDA graph per temperature step,
// whose sweep phase is a single persistent launch over every run's replica groups.  The
// persistent grid is chosen by timing candidate shapes on the batch itself (dry sweeps into
// the spare spin buffers, which leave every run's state untouched).
//
// Each run computes exactly what a single-run context with the same configuration and the
// linear schedule beta_i = i / (n_temps - 1) computes: the kernels are the single-run kernel
// bodies applied through a run table.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "pa_common.cuh"
#include "pa_kernels.h"

namespace {

bool batch_supported_L(int L) { return L >= 4 && L <= 128 && (L % 2) == 0; }

bool register_L(int L) { return pa::batch_group_of(L) != pa::kBatchAnyGroup; }

int rpw_for(int L)
{
    // replicas per replica group: 32 / (lanes per replica), lanes per replica = L / rows per lane
    // (register kernels); the replicas of one warp pass of the shared-memory sweep otherwise
    return register_L(L) ? 32 / (L / pa::rows_per_lane(L)) : pa::any_replicas_per_pass(L);
}

// Replica groups per work item: runs whose groups are small (below 2^14 attempts: small L or
// few sweeps) take 4 to 16 groups per item so that an item holds about 2^16 attempts and the
// per-item cost (work counter, run lookup, sums) stays small; other runs take one.
int ipw_for(int L, int theta)
{
    const long long per_group = (long long)L * L * rpw_for(L) * (theta > 1 ? theta : 1);
    const long long g = (65536 + per_group - 1) / per_group;
    return g < 4 ? 1 : (int)(g > 16 ? 16 : g);
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct RunLayout {
    size_t spins[2], level[2], mag[2], fam[2], work, end;
    pa::Workspace ws;
};

RunLayout layout_run(const pa_run_desc &d, size_t off)
{
    RunLayout r{};
    const size_t bpr = (size_t)pa::bytes_per_replica(d.cfg.L);
    for (int b = 0; b < 2; ++b) {
        r.spins[b] = off;
        off = a256(off + bpr * (size_t)d.cfg.capacity);
    }
    for (int b = 0; b < 2; ++b) {
        r.level[b] = off; off = a256(off + 4 * (size_t)d.cfg.capacity);
        r.mag[b] = off;   off = a256(off + 4 * (size_t)d.cfg.capacity);
        r.fam[b] = off;   off = a256(off + 4 * (size_t)d.cfg.capacity);
    }
    r.ws = pa::plan_workspace(d.cfg.L, d.cfg.capacity);
    r.work = off;
    off = a256(off + r.ws.total);
    r.end = off;
    return r;
}

struct Tables {
    size_t runs, state, ctl, order, item_start, records, desc, end;
};

Tables layout_tables(int n)
{
    Tables t{};
    size_t off = 0;
    t.runs = off;       off = a256(off + sizeof(pa::BatchRun) * (size_t)n);
    t.state = off;      off = a256(off + sizeof(pa::BatchState) * (size_t)n);
    t.ctl = off;        off = a256(off + sizeof(pa::BatchCtl));
    t.order = off;      off = a256(off + sizeof(int) * (size_t)n);
    t.item_start = off; off = a256(off + sizeof(long long) * ((size_t)n + 1));
    t.records = off;    off = a256(off + sizeof(pa_obs) * (size_t)n);
    t.desc = off;       off = a256(off + sizeof(pa::BatchDesc) * (size_t)n);
    t.end = off;
    return t;
}

bool valid_desc(const pa_run_desc &d)
{
    return batch_supported_L(d.cfg.L) && d.cfg.R >= 1 && d.cfg.capacity >= d.cfg.R &&
           d.cfg.capacity <= 2147483647LL && d.cfg.pad == 0 &&
           (d.cfg.update == PA_UPDATE_METROPOLIS || d.cfg.update == PA_UPDATE_HEATBATH) &&
           (d.cfg.resample == PA_RESAMPLE_NEAREST || d.cfg.resample == PA_RESAMPLE_POISSON ||
            d.cfg.resample == PA_RESAMPLE_MULTINOMIAL) &&
           d.n_temps >= 2 && d.theta >= 0 && d.theta <= (1 << 26);
}

}  // namespace

struct pa_batch {
    int n;
    int device, num_sms;
    cudaStream_t user, cs;
    cudaEvent_t ev_in, ev_out;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    char *arena;
    Tables t;
    std::vector<pa_run_desc> desc;
    std::vector<RunLayout> lay;
    int nblk_max, nlev_max;
    int sweep_grid;
    pa_batch_tuning tuning;
    pa::BatchSweepPlan plan;
    std::vector<pa::BatchRun> table;  // host copy of the run table
    int occ[pa::kBatchGroups], occ_all, max_bps;
    int mn_draw_blocks;               // grid of the multinomial draws (0: no multinomial run)
};

namespace {

// Set the sweep phase's shape: plan, and the replica groups per work item in the run table
// (copied to the device; synchronous).
cudaError_t apply_shape(pa_batch *b, int unified, int bps, int scale)
{
    b->plan.unified = unified;
    b->plan.grid_all = b->num_sms * std::min(bps, b->occ_all);
    for (int i = 0; i < b->plan.ngroups; ++i)
        b->plan.grid[i] = register_L(b->plan.L[i]) ? b->num_sms * std::min(bps, b->occ[i]) : b->plan.any_grid;
    for (int i = 0; i < b->n; ++i)
        b->table[(size_t)i].ipw = std::min(16, ipw_for(b->desc[(size_t)i].cfg.L, b->desc[(size_t)i].theta) * scale);
    b->sweep_grid = unified ? b->plan.grid_all : b->num_sms * std::min(bps, b->max_bps);
    return cudaMemcpy(b->arena + b->t.runs, b->table.data(), sizeof(pa::BatchRun) * b->table.size(),
                      cudaMemcpyHostToDevice);
}

// Capture one temperature step of every run into b->graph / b->exec.
cudaError_t capture_step(pa_batch *b)
{
    char *tb = b->arena;
    cudaError_t e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = pa::launch_batch_step(
            reinterpret_cast<const pa::BatchRun *>(tb + b->t.runs), reinterpret_cast<pa::BatchState *>(tb + b->t.state),
            reinterpret_cast<pa::BatchCtl *>(tb + b->t.ctl), reinterpret_cast<const int *>(tb + b->t.order),
            reinterpret_cast<long long *>(tb + b->t.item_start), reinterpret_cast<pa_obs *>(tb + b->t.records), b->n,
            b->nblk_max, b->nlev_max, b->mn_draw_blocks, b->plan, b->cs);
        e = cudaStreamEndCapture(b->cs, &b->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    return e;
}

}  // namespace

static void destroy_plan(pa::BatchSweepPlan &p)
{
    for (int i = 0; i < p.ngroups; ++i) {
        if (p.side[i]) cudaStreamDestroy(p.side[i]);
        if (p.join[i]) cudaEventDestroy(p.join[i]);
    }
    if (p.fork) cudaEventDestroy(p.fork);
    p = pa::BatchSweepPlan{};
}

extern "C" {

pa_status pa_batch_query_sizes(int n_runs, const pa_run_desc *runs, size_t *arena_bytes)
{
    if (n_runs < 1 || !runs || !arena_bytes) return PA_ERR_INVALID_ARG;
    size_t off = layout_tables(n_runs).end;
    for (int i = 0; i < n_runs; ++i) {
        if (!valid_desc(runs[i])) return PA_ERR_INVALID_ARG;
        off = layout_run(runs[i], off).end;
    }
    *arena_bytes = off;
    return PA_OK;
}

pa_status pa_batch_init(int n_runs, const pa_run_desc *runs, void *arena, size_t arena_bytes, void *stream,
                        pa_batch **out)
{
    if (!out) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    size_t need = 0;
    if (pa_batch_query_sizes(n_runs, runs, &need) != PA_OK || !arena || arena_bytes < need ||
        (reinterpret_cast<uintptr_t>(arena) & 255u))
        return PA_ERR_INVALID_ARG;
    pa_batch *b = new (std::nothrow) pa_batch();
    if (!b) return PA_ERR_INVALID_ARG;
    b->n = n_runs;
    b->user = static_cast<cudaStream_t>(stream);
    b->arena = static_cast<char *>(arena);
    b->t = layout_tables(n_runs);
    b->desc.assign(runs, runs + n_runs);
    size_t off = b->t.end;
    b->nblk_max = 1;
    b->nlev_max = 1;
    b->mn_draw_blocks = 0;
    for (int i = 0; i < n_runs; ++i)
        if (runs[i].cfg.resample == PA_RESAMPLE_MULTINOMIAL) {
            const long long blocks = (runs[i].cfg.R + 255) / 256;
            b->mn_draw_blocks = (int)std::max<long long>(b->mn_draw_blocks, std::min<long long>(blocks, 4096));
        }
    for (int i = 0; i < n_runs; ++i) {
        b->lay.push_back(layout_run(runs[i], off));
        off = b->lay.back().end;
        b->nblk_max = std::max(b->nblk_max, (int)b->lay.back().ws.nblk);
        b->nlev_max = std::max(b->nlev_max, runs[i].cfg.L * runs[i].cfg.L + 1);
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete b;
        return PA_ERR_CUDA;
    }

    // host copy of the run table, then step 1 of every run with the single-run kernels
    std::vector<pa::BatchRun> table((size_t)n_runs);
    std::vector<pa::BatchState> state((size_t)n_runs);
    for (int i = 0; i < n_runs; ++i) {
        const pa_run_desc &d = runs[i];
        const RunLayout &L = b->lay[(size_t)i];
        char *base = b->arena;
        char *work = base + L.work;
        pa::DevState *st = reinterpret_cast<pa::DevState *>(work + L.ws.state);
        pa::BatchRun &r = table[(size_t)i];
        std::memset(&r, 0, sizeof(r));
        r.L = d.cfg.L;
        r.theta = d.theta;
        r.n_temps = d.n_temps;
        r.rpw = rpw_for(d.cfg.L);
        r.ipw = ipw_for(d.cfg.L, d.theta);
        r.chunks16 = pa::bytes_per_replica(d.cfg.L) / 16;
        const unsigned int k0 = (unsigned int)(d.cfg.seed & 0xffffffffu), k1 = (unsigned int)(d.cfg.seed >> 32);
        for (int cur = 0; cur < 2; ++cur) {
            const int nxt = cur ^ 1;
            pa::ResampleArgs &a = r.rs[cur];
            a.L = d.cfg.L;
            a.kind = d.cfg.resample;
            a.R_target = d.cfg.R;
            a.capacity = d.cfg.capacity;
            a.k0 = k0;
            a.k1 = k1;
            a.st = st;
            a.hist = reinterpret_cast<int *>(work + L.ws.hist);
            a.fl = reinterpret_cast<int *>(work + L.ws.fl);
            a.thr = reinterpret_cast<unsigned int *>(work + L.ws.thr);
            a.tau = reinterpret_cast<double *>(work + L.ws.tau);
            a.w = reinterpret_cast<double *>(work + L.ws.w);
            a.counts = reinterpret_cast<int *>(work + L.ws.counts);
            a.blocksum = reinterpret_cast<long long *>(work + L.ws.blocksum);
            a.nblk = L.ws.nblk;
            a.wint = reinterpret_cast<unsigned long long *>(work + L.ws.wint);
            a.cdf = reinterpret_cast<unsigned long long *>(work + L.ws.cdf);
            a.spins_src = base + L.spins[cur];
            a.spins_dst = base + L.spins[nxt];
            a.level_src = reinterpret_cast<const int *>(base + L.level[cur]);
            a.mag_src = reinterpret_cast<const int *>(base + L.mag[cur]);
            a.fam_src = reinterpret_cast<const int *>(base + L.fam[cur]);
            a.level_dst = reinterpret_cast<int *>(base + L.level[nxt]);
            a.mag_dst = reinterpret_cast<int *>(base + L.mag[nxt]);
            a.fam_dst = reinterpret_cast<int *>(base + L.fam[nxt]);
            pa::SweepArgs &s = r.sw[cur];
            s.spins = base + L.spins[cur];
            s.level = reinterpret_cast<int *>(base + L.level[cur]);
            s.mag = reinterpret_cast<int *>(base + L.mag[cur]);
            s.fam = reinterpret_cast<int *>(base + L.fam[cur]);
            s.level_snap = reinterpret_cast<int *>(work + L.ws.snap);
            s.hist = reinterpret_cast<int *>(work + L.ws.hist);
            s.st = st;
            s.R_bound = d.cfg.capacity;
            s.k0 = k0;
            s.k1 = k1;
            s.theta = d.theta;
            s.update = d.cfg.update;
            pa::ObsArgs &o = r.obs[cur];
            o.L = d.cfg.L;
            o.R_target = d.cfg.R;
            o.st = st;
            o.hist = reinterpret_cast<int *>(work + L.ws.hist);
            o.fam = reinterpret_cast<int *>(base + L.fam[cur]);
            o.fampart = reinterpret_cast<long long *>(work + L.ws.fampart);
        }
        state[(size_t)i].active = 1;
        state[(size_t)i].step = 0;
        state[(size_t)i].cur = 0;
        state[(size_t)i].status = PA_OK;
        state[(size_t)i].beta = 0.0;
        state[(size_t)i].beta_prev = 0.0;
        // step 1 (simple sampling at beta_0 = 0) and the first measurement
        e = pa::launch_setup(st, d.cfg.R, reinterpret_cast<int *>(work + L.ws.hist), d.cfg.L * d.cfg.L,
                             d.cfg.update, b->user);
        if (e == cudaSuccess) {
            pa::SweepArgs s = r.sw[0];
            s.R_init = d.cfg.R;
            s.R_bound = d.cfg.R;
            s.step = 0;
            s.t0 = 0;
            s.theta = 0;
            e = pa::launch_sweep(d.cfg.L, true, s, b->num_sms, b->user);
        }
        if (e != cudaSuccess) break;
    }
    // runs grouped by lattice size, and within a size the largest per-item cost first
    // (longest-processing-time order)
    std::vector<int> order((size_t)n_runs);
    for (int i = 0; i < n_runs; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int gx = pa::batch_group_of(runs[x].cfg.L), gy = pa::batch_group_of(runs[y].cfg.L);
        if (gx != gy) return gx < gy;
        const double cx = (double)runs[x].cfg.L * runs[x].cfg.L * rpw_for(runs[x].cfg.L) *
                          ipw_for(runs[x].cfg.L, runs[x].theta) * std::max(1, runs[x].theta);
        const double cy = (double)runs[y].cfg.L * runs[y].cfg.L * rpw_for(runs[y].cfg.L) *
                          ipw_for(runs[y].cfg.L, runs[y].theta) * std::max(1, runs[y].theta);
        return cx > cy;
    });
    pa::BatchCtl ctl{};
    ctl.n = n_runs;
    ctl.desc = reinterpret_cast<pa::BatchDesc *>(b->arena + b->t.desc);
    for (int g = 0; g < pa::kBatchGroups; ++g) ctl.pbeg[g] = ctl.pend[g] = 0;
    for (int p = 0; p < n_runs; ++p) {
        const int g = pa::batch_group_of(runs[order[(size_t)p]].cfg.L);
        if (p == 0 || pa::batch_group_of(runs[order[(size_t)p - 1]].cfg.L) != g) ctl.pbeg[g] = p;
        ctl.pend[g] = p + 1;
    }
    // one persistent sweep kernel per size present, on its own side stream
    b->plan = pa::BatchSweepPlan{};
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->plan.fork, cudaEventDisableTiming);
    for (int g = 0; g < pa::kBatchGroups && e == cudaSuccess; ++g) {
        if (ctl.pend[g] == ctl.pbeg[g]) continue;
        const int i = b->plan.ngroups++;
        b->plan.L[i] = runs[order[(size_t)ctl.pbeg[g]]].cfg.L;
        e = cudaStreamCreateWithFlags(&b->plan.side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->plan.join[i], cudaEventDisableTiming);
    }
    char *tb = b->arena;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb + b->t.runs, table.data(), sizeof(pa::BatchRun) * table.size(), cudaMemcpyHostToDevice,
                            b->user);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb + b->t.state, state.data(), sizeof(pa::BatchState) * state.size(),
                            cudaMemcpyHostToDevice, b->user);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb + b->t.ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, b->user);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb + b->t.order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice,
                            b->user);
    const pa::BatchRun *d_runs = reinterpret_cast<const pa::BatchRun *>(tb + b->t.runs);
    pa::BatchState *d_state = reinterpret_cast<pa::BatchState *>(tb + b->t.state);
    pa::BatchCtl *d_ctl = reinterpret_cast<pa::BatchCtl *>(tb + b->t.ctl);
    const int *d_order = reinterpret_cast<const int *>(tb + b->t.order);
    long long *d_items = reinterpret_cast<long long *>(tb + b->t.item_start);
    pa_obs *d_records = reinterpret_cast<pa_obs *>(tb + b->t.records);
    if (e == cudaSuccess) e = pa::launch_batch_record(d_runs, d_state, d_records, n_runs, b->user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->user);  // host tables must outlive the copies

    // autotune the sweep phase on dry sweeps (spare buffers only): one launch over every size
    // or one per size, persistent blocks per SM (each kernel capped by its occupancy), and
    // replica groups per work item (the default count, or twice it)
    b->max_bps = 1;
    b->plan.any_present = 0;
    b->plan.any_kw = 0;
    for (int i = 0; i < n_runs; ++i)
        if (!register_L(runs[i].cfg.L)) {
            b->plan.any_present = 1;
            b->plan.any_kw = std::max(b->plan.any_kw, pa::any_warp_words(runs[i].cfg.L));
        }
    int any_occ = 1;
    if (b->plan.any_present) {
        const size_t smem = pa::batch_any_smem(b->plan.any_kw);
        if (e == cudaSuccess) e = pa::prepare_batch_sweep_any(smem);
        any_occ = pa::batch_any_blocks_per_sm(smem);
        b->plan.any_grid = b->num_sms * any_occ;
    }
    for (int i = 0; i < b->plan.ngroups; ++i) {
        b->occ[i] = register_L(b->plan.L[i]) ? pa::batch_sweep_max_blocks_per_sm(b->plan.L[i]) : any_occ;
        if (register_L(b->plan.L[i])) b->max_bps = std::max(b->max_bps, b->occ[i]);
    }
    b->occ_all = pa::batch_sweep_max_blocks_per_sm(0);
    b->plan.n = n_runs;
    b->table = table;
    struct Shape {
        int unified, bps, scale;
    };
    std::vector<Shape> shapes;
    for (int unified = 0; unified < 2; ++unified)
        for (int bps = 1; bps <= std::min(2, unified ? b->occ_all : b->max_bps); ++bps)
            for (int scale = 1; scale <= 2; scale *= 2) shapes.push_back({unified, bps, scale});
    auto apply = [&](const Shape &sh) -> cudaError_t { return apply_shape(b, sh.unified, sh.bps, sh.scale); };
    std::memset(&b->tuning, 0, sizeof(b->tuning));
    if (e == cudaSuccess) {
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        float best = 1e30f;
        int chosen = 0;
        int dry = 1;
        e = cudaMemcpy(&reinterpret_cast<pa::BatchCtl *>(tb + b->t.ctl)->dry, &dry, sizeof(int), cudaMemcpyHostToDevice);
        for (size_t c = 0; c < shapes.size() && c < 16 && e == cudaSuccess; ++c) {
            e = apply(shapes[c]);
            float ms = 0.f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                e = pa::launch_batch_items(d_runs, d_state, d_ctl, d_order, d_items, n_runs, 0, b->user);
                if (e == cudaSuccess) e = cudaEventRecord(t0, b->user);
                if (e == cudaSuccess) e = pa::launch_batch_sweep(d_ctl, d_items, b->plan, b->user);
                if (e == cudaSuccess) e = cudaEventRecord(t1, b->user);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            }
            pa_batch_shape &cs = b->tuning.cand[b->tuning.n_candidates++];
            cs.unified = shapes[c].unified;
            cs.blocks_per_sm = shapes[c].bps;
            cs.ipw_scale = shapes[c].scale;
            cs.ms = ms;
            if (ms < best) {
                best = ms;
                chosen = (int)c;
            }
        }
        // the single persistent launch is kept unless another shape is more than 2 % faster
        // (the dry-sweep timings of nearby shapes differ by about that much from call to call)
        int best_unified = -1;
        for (int c = 0; c < b->tuning.n_candidates; ++c)
            if (shapes[(size_t)c].unified &&
                (best_unified < 0 || b->tuning.cand[c].ms < b->tuning.cand[best_unified].ms))
                best_unified = c;
        if (best_unified >= 0 && b->tuning.cand[best_unified].ms <= 1.02f * best) chosen = best_unified;
        if (e == cudaSuccess) e = apply(shapes[(size_t)chosen]);
        b->tuning.chosen = chosen;
        b->tuning.chosen_grid = b->sweep_grid;
        dry = 0;
        if (e == cudaSuccess)
            e = cudaMemcpy(&reinterpret_cast<pa::BatchCtl *>(tb + b->t.ctl)->dry, &dry, sizeof(int), cudaMemcpyHostToDevice);
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }

    // capture one temperature step of every run
    if (e == cudaSuccess) e = capture_step(b);
    if (e != cudaSuccess) {
        destroy_plan(b->plan);
        cudaEventDestroy(b->ev_in);
        cudaEventDestroy(b->ev_out);
        cudaStreamDestroy(b->cs);
        delete b;
        return PA_ERR_CUDA;
    }
    *out = b;
    return PA_OK;
}

pa_status pa_batch_step(pa_batch *b)
{
    if (!b) return PA_ERR_INVALID_ARG;
    cudaError_t e = cudaEventRecord(b->ev_in, b->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cs, b->ev_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->cs);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->ev_out, 0);
    return e == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_batch_status(pa_batch *b, int *active_out, int *status_out, long long *step_out)
{
    if (!b) return PA_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->user) != cudaSuccess) return PA_ERR_CUDA;
    std::vector<pa::BatchState> st((size_t)b->n);
    if (cudaMemcpy(st.data(), b->arena + b->t.state, sizeof(pa::BatchState) * st.size(), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return PA_ERR_CUDA;
    for (int i = 0; i < b->n; ++i) {
        if (active_out) active_out[i] = st[(size_t)i].active;
        if (status_out) status_out[i] = st[(size_t)i].status;
        if (step_out) step_out[i] = st[(size_t)i].step;
    }
    return PA_OK;
}

pa_status pa_batch_record(pa_batch *b, void *device_dst)
{
    if (!b || !device_dst) return PA_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(device_dst, b->arena + b->t.records, sizeof(pa_obs) * (size_t)b->n,
                                    cudaMemcpyDeviceToDevice, b->user);
    return e == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_batch_observables(pa_batch *b, pa_obs *host_out)
{
    if (!b || !host_out) return PA_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(host_out, b->arena + b->t.records, sizeof(pa_obs) * (size_t)b->n,
                                    cudaMemcpyDeviceToHost, b->user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->user);
    return e == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_batch_hashes(pa_batch *b, int run, unsigned long long *host_out, long long *count_out)
{
    if (!b || run < 0 || run >= b->n || !host_out || !count_out) return PA_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->user) != cudaSuccess) return PA_ERR_CUDA;
    pa::BatchState st;
    if (cudaMemcpy(&st, b->arena + b->t.state + sizeof(pa::BatchState) * (size_t)run, sizeof(st),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return PA_ERR_CUDA;
    const RunLayout &L = b->lay[(size_t)run];
    const pa_run_desc &d = b->desc[(size_t)run];
    char *work = b->arena + L.work;
    const pa::DevState *dst = reinterpret_cast<const pa::DevState *>(work + L.ws.state);
    unsigned long long *dev = reinterpret_cast<unsigned long long *>(work + L.ws.hashes);
    cudaError_t e = pa::launch_hashes(d.cfg.L, b->arena + L.spins[st.cur], d.cfg.capacity, dst, dev, b->user);
    long long R = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->user);
    if (e == cudaSuccess) e = cudaMemcpy(&R, &dst->R_cur, sizeof(R), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(host_out, dev, sizeof(unsigned long long) * (size_t)R, cudaMemcpyDeviceToHost);
    *count_out = R;
    return e == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_batch_set_shape(pa_batch *b, const pa_batch_shape *shape)
{
    if (!b || !shape || (shape->unified != 0 && shape->unified != 1) || shape->blocks_per_sm < 1 ||
        shape->blocks_per_sm > 32 || shape->ipw_scale < 1 || shape->ipw_scale > 16)
        return PA_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->cs) != cudaSuccess || cudaStreamSynchronize(b->user) != cudaSuccess)
        return PA_ERR_CUDA;
    if (apply_shape(b, shape->unified, shape->blocks_per_sm, shape->ipw_scale) != cudaSuccess) return PA_ERR_CUDA;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (capture_step(b) != cudaSuccess) return PA_ERR_CUDA;
    b->tuning.chosen = -1;
    b->tuning.chosen_grid = b->sweep_grid;
    return PA_OK;
}

pa_status pa_batch_get_tuning(const pa_batch *b, pa_batch_tuning *out)
{
    if (!b || !out) return PA_ERR_INVALID_ARG;
    *out = b->tuning;
    return PA_OK;
}

void pa_batch_destroy(pa_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->cs);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    destroy_plan(b->plan);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
    cudaStreamDestroy(b->cs);
    delete b;
}

}  // extern "C"
