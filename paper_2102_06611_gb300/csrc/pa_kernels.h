// pa_kernels.h -- argument blocks and launchers of the library's kernels (internal).
#pragma once

#include <mutex>

#include <cuda_runtime.h>

#include "pa.h"

namespace pa {

struct DevState;

// Runs a one-time set-up step (e.g. raising a kernel's dynamic shared-memory limit, an
// attribute each device keeps separately) once per device: the device current at the call
// selects the flag.  Thread safe.
class PerDeviceOnce {
public:
    template <class F>
    cudaError_t operator()(F &&f)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kDevices) return f();
        std::lock_guard<std::mutex> lock(mu_);
        if (done_[dev]) return cudaSuccess;
        e = f();
        if (e == cudaSuccess) done_[dev] = true;
        return e;
    }

private:
    static constexpr int kDevices = 64;
    std::mutex mu_;
    bool done_[kDevices] = {};
};

// Workspace layout (byte offsets, all 256-byte aligned), computed by plan_workspace().
struct Workspace {
    size_t state;       // DevState
    size_t hist;        // int32[N + 1]   level histogram of the current population
    size_t fl;          // int32[N + 1]   floor(tau_hat_k)
    size_t thr;         // uint32[N + 1]  floor(frac(tau_hat_k) 2^32)
    size_t tau;         // double[N + 1]  tau_hat_k
    size_t w;           // double[N + 1]  w_k
    size_t counts;      // int32[capacity] copy numbers r_j of the last resampling
    size_t blocksum;    // int64[nblk]    per-block sums of r_j, then exclusive offsets
    size_t fampart;     // int64[2 * kFamBlocks] family partial sums
    size_t obs;         // pa_obs          record slot used by pa_observables
    size_t hashes;      // uint64[capacity]
    size_t stage;       // uint32[kStageReplicas * L * ceil(L/32)] export staging
    size_t occ_k;       // int32[N + 1]   occupied levels, ascending (schedule proposals)
    size_t occ_h;       // int32[N + 1]   their counts
    size_t occ_w;       // double[N + 1]  reweighting factors at a trial step
    size_t occ_t;       // double[N + 1]  overlap terms at a trial step
    size_t feat;        // float[32]      learned-schedule features (raw, standardised), then a uint64 zero count
    size_t snap;        // int32[capacity] levels at the start of the temperature step
    size_t ana_blk;     // int64[4 * kMaxAnaBlocks] analysis block sums
    size_t ana_sizes;   // int32[capacity + 1]     family-size histogram (entry 0: largest size)
    size_t ana_out;     // pa_analysis
    size_t wint;        // uint64[N + 1]  multinomial: integer weights floor(w_k 2^32)
    size_t cdf;         // uint64[capacity] multinomial: running sum of the parents' weights
    size_t search;      // SearchState        temperature-step search
    size_t hist_before; // int32[N + 1]   sharded population: level histogram of the shards before this one
    size_t total;
    long long nblk;     // blocks of the copy-count / copy kernels
};

constexpr int kCountThreads = 256;
constexpr int kCountItems = 4;                              // parents per thread
constexpr int kCountBlockItems = kCountThreads * kCountItems; // parents per block
constexpr int kFamBlocks = 512;
constexpr long long kStageReplicas = 4096;
constexpr int kMaxAnaBlocks = 1024;

Workspace plan_workspace(int L, long long capacity);

struct SweepArgs {
    void *spins;            // current spin buffer (updated in place)
    int *level;
    int *mag;
    int *fam;               // written only by the init kernel
    int *level_snap;        // levels at the start of the temperature step (sweep kernel)
    int *hist;
    DevState *st;
    long long R_init;       // population size for the init kernel
    long long R_bound;      // host-side upper bound on R (grid sizing only)
    unsigned int k0, k1;    // Philox key (seed)
    unsigned int step;      // temperature index i
    int t0;                 // sweeps already done at this step (sweep numbering offset)
    int theta;
    int update;             // pa_update_kind (the init kernel ignores it)
    // the run's acceptance thresholds at the current beta, computed on the host with the
    // same binary64 arithmetic as DevState::T4 / T8 (k_sweep reads them from its
    // parameters, where they are warp-uniform operands, and checks them against DevState)
    unsigned long long T4, T8;
    // global slot of local replica 0: a population split over several shards by contiguous slot
    // ranges keys every random number (and the initial family id) by the global slot (0 for a
    // population held whole)
    unsigned int slot_base;
};

cudaError_t launch_sweep(int L, bool init, const SweepArgs &a, int num_sms, cudaStream_t s);
// the sizes with a register-resident kernel template (pa_sweep.cuh); launch_sweep forwards
// every other even 4 <= L <= 128 to the shared-memory kernel of pa_sweep_any.cu
bool sweep_has_template(int L);
cudaError_t launch_sweep_any(int L, bool init, const SweepArgs &a, int num_sms, cudaStream_t s);
// the heatbath sweep (pa_sweep_hb.cu); launch_sweep forwards to it for a.update = heatbath
cudaError_t launch_sweep_hb(int L, const SweepArgs &a, int num_sms, cudaStream_t s);

struct ResampleArgs {
    int L;
    int kind;
    long long R_target;
    long long capacity;
    double beta_prev, beta_new;
    unsigned int step;
    unsigned int k0, k1;
    DevState *st;
    const int *hist;
    int *fl;
    unsigned int *thr;
    double *tau;
    double *w;
    int *counts;
    long long *blocksum;
    long long nblk;
    unsigned long long *wint;  // multinomial only
    unsigned long long *cdf;   // multinomial only
    const void *spins_src;
    void *spins_dst;
    const int *level_src, *mag_src, *fam_src;
    int *level_dst, *mag_dst, *fam_dst;
    // sharded population: the histogram is the whole population's (DevState::R_glob parents,
    // used for ln Q_i) and local parent j has the global index parent_base + j
    int sharded;
    unsigned int parent_base;
    // sharded multinomial resampling: level histogram of the parents of the shards before this
    // one (their weight sum places this shard's parents in the whole population's running sum)
    const int *hist_before;
    // the replica copy writes only children [win_lo, win_lo + win_n) (local child indices, in
    // tree order) to destination index child - win_lo; win_n = 0: every child, at its index
    long long win_lo, win_n;
};

cudaError_t launch_resample(const ResampleArgs &a, cudaStream_t s);
cudaError_t launch_copy_numbers(const ResampleArgs &a, cudaStream_t s);
cudaError_t launch_copy(const ResampleArgs &a, cudaStream_t s);
cudaError_t launch_thresholds(DevState *st, double beta, cudaStream_t s);
cudaError_t launch_zero_measure(DevState *st, int *hist, int N, cudaStream_t s);
cudaError_t launch_setup(DevState *st, long long R, int *hist, int N, int update, cudaStream_t s);

struct ObsArgs {
    int L;
    long long R_target;
    long long step;
    double beta, dbeta;
    int theta;
    DevState *st;
    const int *hist;
    const int *fam;
    long long *fampart;
    pa_obs *dst;
    int glob;               // sharded population: R, family counts and sums from the combined state
};

cudaError_t launch_observables(const ObsArgs &a, cudaStream_t s);

// Sharded populations: one shard's summary (level histogram, exact sums, family edges) and
// the combination of all shards' summaries into the whole population's state.
constexpr int kShardExtra = 16;  // int64 entries after the N + 1 histogram entries
cudaError_t launch_shard_summary(const DevState *st, const int *hist, const int *fam, const long long *fampart,
                                 int N, long long *out, cudaStream_t s);
cudaError_t launch_shard_combine(DevState *st, int *hist, int *hist_before, long long slot_base, int N,
                                 const long long *all, int n_shards, cudaStream_t s);
cudaError_t launch_set_population(DevState *st, long long R, cudaStream_t s);

// Weighted average over independent runs' records (pa_analysis.cu).
cudaError_t launch_weighted(const pa_obs *rec, int M, int mode, pa_weighted *out, cudaStream_t s);

// Population analysis (pa_analysis.cu): block sums, family-size histogram, binary64 results.
cudaError_t launch_analysis(const DevState *st, const int *level, const int *mag, const int *fam, int N,
                            double beta, int n, long long capacity, long long *blk, int *sizes, pa_analysis *out,
                            cudaStream_t s);

// Adaptive temperature step: search on dbeta for the histogram overlap (pa_schedule.cu).
struct BisectArgs {
    int L;
    DevState *st;
    const int *hist;
    int *occ_k, *occ_h;
    double *occ_w, *occ_t;
    double beta, beta_final, dbeta_max, alpha_target;
    int iters;
    int use_prop;        // first try the step in st->dbeta_prop against alpha_floor
    double alpha_floor;
};

constexpr int kBisectIters = 48;

// State of one search for the next temperature step (device workspace, pa_schedule.cu).
constexpr int kSearchK = 64;  // points per round: the bracket shrinks by 64 per round
struct SearchBracket {
    double lo, hi, a_lo;
};
struct SearchState {
    int nocc, kmin, done, source;
    long long R;
    double invR;                         // 1 / R (binary64)
    double hi0, dbeta, alpha;
    SearchBracket br[2];                 // bracket of the last two rounds
    double alpha_pts[2][kSearchK];       // overlaps at the points of the last two rounds
};
cudaError_t launch_bisect(const BisectArgs &a, SearchState *ss, cudaStream_t s);
cudaError_t launch_families(const DevState *st, const int *fam, long long *fampart, cudaStream_t s);

// Learned schedule (pa_mlp.cu).
struct FeatureArgs {
    int L;
    const DevState *st;
    const int *hist;
    const long long *fampart;
    const int *counts;
    double beta, dbeta_prev, theta_ratio_prev, alpha_prev;
    const float *norm;   // x_mean[12], x_std[12], y_mean[2], y_std[2] (may be null: raw only)
    float *raw;          // 12 features
    float *x;            // 12 standardised features
    unsigned long long *zeros;  // scratch: parents with zero copies (counted by many blocks)
    long long capacity;  // replicas the buffers hold (grid of the zero count)
};

cudaError_t launch_features(const FeatureArgs &a, cudaStream_t s);
cudaError_t launch_mlp_propose(const unsigned short *P, const float *norm, const float *raw, const float *x, int L,
                               double dbeta_max, int theta_max, DevState *st, cudaStream_t s);

// ------------------------------------------------------------------------------ batches
// Many independent runs advance one temperature step per replay of a captured graph.  Each
// run keeps the single-run layout (its own buffers and workspace); the kernels below take a
// run table and use blockIdx.y (or a work item) to pick the run.
struct BatchRun {
    ResampleArgs rs[2];   // resampling arguments with `cur` = 0 / 1 (beta, step patched per step)
    ObsArgs obs[2];       // record arguments with `cur` = 0 / 1
    SweepArgs sw[2];      // sweep arguments with `cur` = 0 / 1
    int L, theta, n_temps, rpw;
    int chunks16;
    int ipw;              // replica groups (of rpw replicas) per work item
};

struct BatchState {       // per run, mutable
    int active;           // 1 while beta < 1 and no error
    int step;             // temperature index i
    int cur;              // buffers holding the current population
    int status;           // pa_status of the run
    double beta, beta_prev;
};

// Lattice sizes of batches, one persistent sweep kernel each.
// Lattice-size groups of a batch: one per size with a register sweep kernel, and one for
// every other even L (the shared-memory sweep).
constexpr int kBatchGroups = 10;
constexpr int kBatchAnyGroup = kBatchGroups - 1;
__host__ __device__ constexpr int batch_group_of(int L)
{
    return L == 4 ? 0 : L == 8 ? 1 : L == 12 ? 2 : L == 16 ? 3 : L == 24 ? 4 : L == 32 ? 5 : L == 48 ? 6
           : L == 64 ? 7 : L == 128 ? 8 : kBatchAnyGroup;
}

// What the sweep of one run needs for the current step, per order position, written by
// k_b_items just before the sweep phase: a work item finds it with one load after the search
// for its position (instead of a chain of loads through the run table and the run's state).
struct BatchDesc {
    SweepArgs a;          // current buffers; step, t0 = 0, theta and the thresholds T4 / T8 set
    const void *spare;    // the other spin buffer (dry sweeps write there)
    long long item0;      // the run's first work item
    long long R;          // the run's population size R_i
    int ipw, L;
};

// Order position of a work item: the largest p in [lo, hi) with item_start[p] <= item
// (read-only loads: item_start does not change during the sweep phase).
__device__ __forceinline__ int item_position(const long long *item_start, long long item, int lo, int hi)
{
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(item_start + mid) <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

struct BatchCtl {
    unsigned long long next_item;  // work counter (unused by the per-size kernels)
    long long total_items;
    int n;
    int dry;              // autotuning: sweep into the spare buffer, measure nothing
    // per lattice-size group g: runs at order positions [pbeg[g], pend[g]) (fixed at
    // initialisation), their work items [begin[g], end[g]) and the group's work counter
    int pbeg[kBatchGroups], pend[kBatchGroups];
    long long begin[kBatchGroups], end[kBatchGroups];
    unsigned long long next[kBatchGroups];
    BatchDesc *desc;      // per order position (n entries, in the batch's table memory)
};

// Host plan of the sweep phase: one persistent kernel per lattice size present, launched on
// side streams forked from (and joined back into) the step's stream.
struct BatchSweepPlan {
    int ngroups;
    int L[kBatchGroups];
    int grid[kBatchGroups];
    cudaStream_t side[kBatchGroups];
    cudaEvent_t fork, join[kBatchGroups];
    // one launch over every size (k_b_sweep_all, grid_all blocks) instead of one per size
    int unified, grid_all, n;
    // the runs without a register kernel (group kBatchAnyGroup): present, warp staging words
    int any_present, any_kw, any_grid;
};

cudaError_t launch_batch_step(const BatchRun *runs, BatchState *state, BatchCtl *ctl, const int *order,
                              long long *item_start, pa_obs *records, int n, int nblk_max, int nlev_max, int mn_draw_blocks,
                              const BatchSweepPlan &plan, cudaStream_t s);
cudaError_t launch_batch_items(const BatchRun *runs, BatchState *state, BatchCtl *ctl, const int *order,
                               long long *item_start, int n, int dry, cudaStream_t s);
cudaError_t launch_batch_sweep(BatchCtl *ctl, const long long *item_start, const BatchSweepPlan &plan, cudaStream_t s);
cudaError_t launch_batch_record(const BatchRun *runs, BatchState *state, pa_obs *records, int n,
                                cudaStream_t s);
int batch_sweep_max_blocks_per_sm(int L);

// Batched shared-memory sweep (pa_sweep_any.cu) for the runs whose L has no register kernel:
// replicas per warp pass, the staging words a warp needs for L, dynamic shared memory per block
// for a largest warp need of max_kw words (the limit is raised by prepare_batch_sweep_any, to
// be called before any capture), resident blocks per SM, and the persistent launch.
int any_replicas_per_pass(int L);
int any_warp_words(int L);
size_t batch_any_smem(int max_kw);
cudaError_t prepare_batch_sweep_any(size_t smem);
int batch_any_blocks_per_sm(size_t smem);
cudaError_t launch_batch_sweep_any(BatchCtl *ctl, const long long *item_start, int grid, int max_kw, cudaStream_t s);

cudaError_t launch_hashes(int L, const void *spins, long long R, const DevState *st,
                          unsigned long long *out, cudaStream_t s);
cudaError_t launch_export(int L, const void *spins, long long first, long long count,
                          unsigned int *out, cudaStream_t s);

}  // namespace pa
