// pa_shard.cu -- one population split over several shards (devices or processes) by contiguous
// ranges of replica slots (arXiv:2102.06611, Sec. II).
//
// Sweeps and measurements are local to a shard.  The method couples the replicas once per
// temperature step, through the normalisation of the weights (Eq. Q and Eq. taus need the
// whole population's energy histogram and size) and through the placement of the children in
// tree order.  A shard therefore publishes a summary after each measurement: its level
// histogram, its exact integer sums, and the family ids and run lengths at its two ends.  Every
// shard combines all summaries, in slot order, into the whole population's histogram, sums and
// family statistics; being integers, the combination is exact and identical on every shard,
// so the binary64 tables that follow are too.  The summary layout (int64 entries) is
//   [0, N]        level histogram h_k
//   N+1 + 0       replicas of the shard
//   N+1 + 1..2    sum |M|, sum M^2
//   N+1 + 3..7    sum k0, k0^2, k1, k1^2, k0 k1 (levels at the step start and now)
//   N+1 + 8..9    family id of the first replica, length of its run of equal ids
//   N+1 + 10..11  family id of the last replica, length of its run
//   N+1 + 12..13  number of families (runs) and sum of run length^2 within the shard
//   N+1 + 14..15  zero
#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {
namespace {

constexpr int kShardThreads = 1024;

__device__ __forceinline__ long long block_sum_ll(long long v, long long *part)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kShardThreads / 32; ++i) t += part[i];
    __syncthreads();
    return t;  // valid in thread 0
}

// Length of the run of ids equal to fam[from] going in direction dir (+1 or -1), by
// galloping then bisection (ids are sorted, so equal ids are contiguous).
__device__ long long run_length(const int *fam, long long R, long long from, int dir)
{
    const int f = fam[from];
    long long lo = 0, step = 1;  // offsets: fam[from + dir * lo] == f
    while (true) {
        const long long t = lo + step;
        const long long idx = from + dir * t;
        if (idx < 0 || idx >= R || fam[idx] != f) break;
        lo = t;
        step <<= 1;
    }
    long long hi = lo + step;  // first offset known (or assumed at the boundary) to differ
    while (hi - lo > 1) {
        const long long mid = lo + (hi - lo) / 2;
        const long long idx = from + dir * mid;
        if (idx >= 0 && idx < R && fam[idx] == f) lo = mid;
        else hi = mid;
    }
    return lo + 1;
}

__global__ void __launch_bounds__(kShardThreads) k_shard_summary(const DevState *st, const int *hist, const int *fam,
                                                                 const long long *fampart, int N, long long *out)
{
    __shared__ long long part[kShardThreads / 32];
    for (int k = threadIdx.x; k <= N; k += kShardThreads) out[k] = hist[k];
    long long fc = 0, f2 = 0;
    for (int b = threadIdx.x; b < kFamBlocks; b += kShardThreads) {
        fc += fampart[2 * b];
        f2 += fampart[2 * b + 1];
    }
    fc = block_sum_ll(fc, part);
    f2 = block_sum_ll(f2, part);
    if (threadIdx.x != 0) return;
    long long *x = out + N + 1;
    const long long R = st->R_cur;
    x[0] = R;
    x[1] = (long long)st->sum_absM;
    x[2] = (long long)st->sum_M2;
    x[3] = st->c0;
    x[4] = st->c00;
    x[5] = st->c1;
    x[6] = st->c11;
    x[7] = st->c01;
    if (R > 0) {
        x[8] = fam[0];
        x[9] = run_length(fam, R, 0, +1);
        x[10] = fam[R - 1];
        x[11] = run_length(fam, R, R - 1, -1);
    } else {
        x[8] = x[9] = x[10] = x[11] = 0;
    }
    x[12] = R > 0 ? fc : 0;
    x[13] = R > 0 ? f2 : 0;
    x[14] = x[15] = 0;
}

// All shards' summaries (n_shards rows of N + 1 + kShardExtra, in slot order) into the
// whole population's state: h_k summed, the exact sums summed, and the families merged where
// one run of equal ids crosses shard boundaries (a run may span several shards).  The rows
// that end at or below this shard's first slot (slot_base) are the shards before it: their
// summed histogram goes to hist_before (multinomial resampling places this shard's parents
// in the whole population's running weight sum with it).
__global__ void __launch_bounds__(kShardThreads) k_shard_combine(DevState *st, int *hist, int *hist_before,
                                                                 long long slot_base, int N, const long long *all,
                                                                 int n_shards)
{
    __shared__ long long part[kShardThreads / 32];
    const int V = N + 1 + kShardExtra;
    long long tot = 0;
    for (int k = threadIdx.x; k <= N; k += kShardThreads) {
        long long h = 0, hb = 0, end = 0;
        for (int s = 0; s < n_shards; ++s) {
            const long long v = all[(size_t)s * V + k];
            end += all[(size_t)s * V + N + 1];
            h += v;
            if (end <= slot_base) hb += v;
        }
        hist[k] = (int)h;
        hist_before[k] = (int)hb;
        tot += h;
    }
    tot = block_sum_ll(tot, part);
    if (threadIdx.x != 0) return;
    long long R = 0, sums[7] = {0, 0, 0, 0, 0, 0, 0};
    long long f = 0, s2 = 0, open_id = 0, open_len = 0;
    bool open = false, own = false;
    for (int s = 0; s < n_shards; ++s) {
        const long long *x = all + (size_t)s * V + N + 1;
        const long long Rs = x[0];
        if (R == slot_base && Rs == st->R_cur) own = true;  // this shard's own row
        R += Rs;
        for (int i = 0; i < 7; ++i) sums[i] += x[1 + i];
        if (Rs <= 0) continue;
        // the shard's first run continues the open run, or starts a new one
        if (open && open_id == x[8]) {
            open_len += x[9];
        } else {
            if (open) {
                f += 1;
                s2 += open_len * open_len;
            }
            open = true;
            open_id = x[8];
            open_len = x[9];
        }
        if (x[12] > 1) {  // the first run ends inside the shard: close it, add the inner runs
            f += 1;
            s2 += open_len * open_len;
            f += x[12] - 2;
            s2 += x[13] - x[9] * x[9] - x[11] * x[11];
            open_id = x[10];
            open_len = x[11];
        }
    }
    if (open) {
        f += 1;
        s2 += open_len * open_len;
    }
    st->R_glob = R;
    st->sum_absM = (unsigned long long)sums[0];
    st->sum_M2 = (unsigned long long)sums[1];
    st->c0 = sums[2];
    st->c00 = sums[3];
    st->c1 = sums[4];
    st->c11 = sums[5];
    st->c01 = sums[6];
    st->fam_count = f;
    st->fam_size2 = s2;
    // inconsistent summaries (not in slot order, or without this shard's row) or no replicas
    if (tot != R || R < 1 || !own) set_error(st, PA_ERR_NUMERIC);
}

__global__ void k_set_population(DevState *st, long long R)
{
    st->R_cur = R;
}

}  // namespace

cudaError_t launch_shard_summary(const DevState *st, const int *hist, const int *fam, const long long *fampart,
                                 int N, long long *out, cudaStream_t s)
{
    k_shard_summary<<<1, kShardThreads, 0, s>>>(st, hist, fam, fampart, N, out);
    return cudaGetLastError();
}

cudaError_t launch_shard_combine(DevState *st, int *hist, int *hist_before, long long slot_base, int N,
                                 const long long *all, int n_shards, cudaStream_t s)
{
    k_shard_combine<<<1, kShardThreads, 0, s>>>(st, hist, hist_before, slot_base, N, all, n_shards);
    return cudaGetLastError();
}

cudaError_t launch_set_population(DevState *st, long long R, cudaStream_t s)
{
    k_set_population<<<1, 1, 0, s>>>(st, R);
    return cudaGetLastError();
}

}  // namespace pa
