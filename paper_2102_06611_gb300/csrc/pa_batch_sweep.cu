// pa_batch_sweep.cu -- the persistent sweep kernels of batches (pa_batch.cu): the
// single-run sweep arithmetic (pa_sweep.cuh) applied to work items of many runs.
#include "pa_sweep.cuh"

// Block shape of the batched sweep kernels: PA_BATCH_THREADS threads, at least
// PA_BATCH_MIN_BLOCKS resident blocks per SM (so at most 65536 / (threads x blocks) registers).
// One block of 384 per SM (12 warps, at most 170 registers) was measured best on the 64-run
// mixed workload: 2.87 ms per dry sweep against 2.99 (512 x 1) and 3.02 (256 x 2).
#ifndef PA_BATCH_THREADS
#define PA_BATCH_THREADS 384
#endif
#ifndef PA_BATCH_MIN_BLOCKS
#define PA_BATCH_MIN_BLOCKS 1
#endif
constexpr int kBatchWarps = PA_BATCH_THREADS / 32;

namespace pa {

// ------------------------------------------------------------------------------ batches
// One persistent launch per lattice size present sweeps the active runs of that size (the
// launches run concurrently on side streams): warps take work items (ipw consecutive
// replica groups of one run) from the size's counter, largest items first (runs are
// ordered by cost within a size); an item finds its run's sweep descriptor (BatchDesc,
// written by k_b_items for this step) by a search of the item offsets and one load, which
// measured 3 % faster at L = 32, 64 than following the run table and the run's state.  The
// per-replica arithmetic
// is exactly the single-run kernel's, with the histogram and sums going to the run's own
// workspace: level counts aggregated over the warp, the seven exact sums once per item.
// A warp's tie queue in the kernel's dynamic shared memory (inv: heatbath only).
struct TqBuf {
    unsigned long long *eq, *a4, *inv;
    unsigned int *code;
};

template <int L, bool HB>
__device__ __forceinline__ TieQueue<typename Geo<L>::W> tie_queue(const TqBuf &qb)
{
    using W = typename Geo<L>::W;
    return TieQueue<W>{reinterpret_cast<W *>(qb.eq), reinterpret_cast<W *>(qb.a4),
                       HB ? reinterpret_cast<W *>(qb.inv) : nullptr, qb.code};
}

template <int L, bool HB>
__device__ __forceinline__ void batch_group(const SweepArgs &a, const void *spare, long long g, long long R, int lane,
                                            int dry, const TqBuf &qb, const unsigned int *rk0, const unsigned int *rk1,
                                            unsigned long long *v)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    constexpr int N = Gm::N, G = Gm::G, RPW = Gm::RPW, RPL = Gm::RPL;
    const int q = lane & (G - 1);
    const int sub = lane / G;
    const int r0 = q * RPL;
    const long long j = g * RPW + sub;
    const bool active = j < R;
    const Accept<W> ac = make_accept<L>(a.T4, a.T8);
    W A[RPL], B[RPL];
    W *rep = reinterpret_cast<W *>(a.spins) + (size_t)(active ? j : 0) * (2 * L);
    if (active) load_rows<L>(rep, r0, A, B);
    else {
#pragma unroll
        for (int i = 0; i < RPL; ++i) { A[i] = 0; B[i] = 0; }
    }
    const TieQueue<W> tq = tie_queue<L, HB>(qb);
    sweep_rows<L, HB>(A, B, r0, lane, (unsigned int)j, (unsigned int)(g * RPW), 0, a.theta, a.step, rk0, rk1, ac, tq);
    int anti, ups;
    measure_rows<L>(A, B, r0, lane, anti, ups);
    anti = group_sum<G>(anti);
    ups = group_sum<G>(ups);
    int level = -1;
    if (active) {
        if (dry) {
            store_rows<L>(reinterpret_cast<W *>(const_cast<void *>(spare)) + (size_t)j * (2 * L), r0, A, B);
        } else {
            if (a.theta > 0) store_rows<L>(rep, r0, A, B);
            if (q == 0) {
                level = anti >> 1;
                const int M = 2 * ups - N;
                const unsigned long long k0 = (unsigned long long)a.level[j];
                const unsigned long long k1 = (unsigned long long)level;
                a.level_snap[j] = (int)k0;
                a.level[j] = level;
                a.mag[j] = M;
                v[0] += (unsigned long long)(M < 0 ? -M : M);
                v[1] += (unsigned long long)((long long)M * M);
                v[2] += k0;
                v[3] += k0 * k0;
                v[4] += k1;
                v[5] += k1 * k1;
                v[6] += k0 * k1;
            }
        }
    }
    if constexpr (RPW >= 8) {
        // many replicas per warp: one atomic per distinct level
        const unsigned int grp = __match_any_sync(0xffffffffu, level);
        if (level >= 0 && lane == __ffs((int)grp) - 1) atomicAdd(&a.hist[level], __popc(grp));
    } else if (level >= 0) {
        atomicAdd(&a.hist[level], 1);
    }
}

// Items of one group (ipw = 1) take this form, which nvcc compiles to faster code for them
// than the general loop below (measured).
template <int L, bool HB>
__device__ __forceinline__ void batch_item_single(const SweepArgs &a, const void *spare, long long g, long long R,
                                                  int lane, int dry, const TqBuf &qb)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    constexpr int N = Gm::N, G = Gm::G, RPW = Gm::RPW, RPL = Gm::RPL;
    const int q = lane & (G - 1);
    const int sub = lane / G;
    const int r0 = q * RPL;
    const long long j = g * RPW + sub;
    const bool active = j < R;
    unsigned int rk0[10], rk1[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        rk0[i] = a.k0 + (unsigned int)i * kPhiloxW0;
        rk1[i] = a.k1 + (unsigned int)i * kPhiloxW1;
    }
    const Accept<W> ac = make_accept<L>(a.T4, a.T8);
    W A[RPL], B[RPL];
    W *rep = reinterpret_cast<W *>(a.spins) + (size_t)(active ? j : 0) * (2 * L);
    if (active) load_rows<L>(rep, r0, A, B);
    else {
#pragma unroll
        for (int i = 0; i < RPL; ++i) { A[i] = 0; B[i] = 0; }
    }
    const TieQueue<W> tq = tie_queue<L, HB>(qb);
    sweep_rows<L, HB>(A, B, r0, lane, (unsigned int)j, (unsigned int)(g * RPW), 0, a.theta, a.step, rk0, rk1, ac, tq);
    int anti, ups;
    measure_rows<L>(A, B, r0, lane, anti, ups);
    anti = group_sum<G>(anti);
    ups = group_sum<G>(ups);
    unsigned long long v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (active) {
        if (dry) {
            store_rows<L>(reinterpret_cast<W *>(const_cast<void *>(spare)) + (size_t)j * (2 * L), r0, A, B);
        } else {
            if (a.theta > 0) store_rows<L>(rep, r0, A, B);
            if (q == 0) {
                const int level = anti >> 1;
                const int M = 2 * ups - N;
                const unsigned long long k0 = (unsigned long long)a.level[j];
                const unsigned long long k1 = (unsigned long long)level;
                a.level_snap[j] = (int)k0;
                a.level[j] = level;
                a.mag[j] = M;
                atomicAdd(&a.hist[level], 1);
                v[0] = (unsigned long long)(M < 0 ? -M : M);
                v[1] = (unsigned long long)((long long)M * M);
                v[2] = k0;
                v[3] = k0 * k0;
                v[4] = k1;
                v[5] = k1 * k1;
                v[6] = k0 * k1;
            }
        }
    }
    // all replicas of the item belong to one run: one atomic per sum and item
#pragma unroll
    for (int i = 0; i < 7; ++i) v[i] = group_sum<32>(v[i]);
    if (lane == 0 && !dry) {
        atomicAdd(&a.st->sum_absM, v[0]);
        atomicAdd(&a.st->sum_M2, v[1]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c0), v[2]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c00), v[3]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c1), v[4]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c11), v[5]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c01), v[6]);
    }
}

template <int L, bool HB>
__device__ __forceinline__ void batch_item(const SweepArgs &a, const void *spare, long long item, int ipw, long long R,
                                           int lane, int dry, const TqBuf &qb)
{
    constexpr int RPW = Geo<L>::RPW;
    if (ipw == 1) {  // uniform over the warp
        batch_item_single<L, HB>(a, spare, item, R, lane, dry, qb);
        return;
    }
    unsigned int rk0[10], rk1[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        rk0[i] = a.k0 + (unsigned int)i * kPhiloxW0;
        rk1[i] = a.k1 + (unsigned int)i * kPhiloxW1;
    }
    unsigned long long v[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll 1
    for (int k = 0; k < ipw; ++k) {
        const long long g = item * ipw + k;
        if (g * RPW >= R) break;  // uniform over the warp
        batch_group<L, HB>(a, spare, g, R, lane, dry, qb, rk0, rk1, v);
    }
    // every replica of the item belongs to one run: one atomic per sum and item
#pragma unroll
    for (int i = 0; i < 7; ++i) v[i] = group_sum<32>(v[i]);
    if (lane == 0 && !dry) {
        atomicAdd(&a.st->sum_absM, v[0]);
        atomicAdd(&a.st->sum_M2, v[1]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c0), v[2]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c00), v[3]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c1), v[4]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c11), v[5]);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c01), v[6]);
    }
}

// The run's spin update decides the instantiation (uniform over the warp).
template <int L>
__device__ __forceinline__ void batch_item_update(const BatchDesc &d, long long item, int lane, int dry,
                                                  const TqBuf &qb)
{
    if (d.a.update == PA_UPDATE_HEATBATH) batch_item<L, true>(d.a, d.spare, item, d.ipw, d.R, lane, dry, qb);
    else batch_item<L, false>(d.a, d.spare, item, d.ipw, d.R, lane, dry, qb);
}

// Tie queues of the kBatchWarps warps of a block of a kernel with TQ entries per warp:
// eq, a4, inv (8-byte entries) and code (4-byte entries), in dynamic shared memory.
constexpr size_t tq_smem_bytes(int TQ) { return (size_t)kBatchWarps * TQ * (3 * 8 + 4); }

__device__ __forceinline__ TqBuf warp_tq(unsigned long long *sh, int TQ)
{
    const int wib = threadIdx.x >> 5;
    TqBuf qb;
    qb.eq = sh + (size_t)wib * TQ;
    qb.a4 = sh + (size_t)kBatchWarps * TQ + (size_t)wib * TQ;
    qb.inv = sh + (size_t)2 * kBatchWarps * TQ + (size_t)wib * TQ;
    qb.code = reinterpret_cast<unsigned int *>(sh + (size_t)3 * kBatchWarps * TQ) + (size_t)wib * TQ;
    return qb;
}

// Persistent sweep over the work items of the runs with lattice size L (group g): warps
// take items from the group's counter; the item's run is found by bisection over the
// group's order positions.
template <int L>
__global__ void __launch_bounds__(PA_BATCH_THREADS, PA_BATCH_MIN_BLOCKS) k_b_sweep(BatchCtl *ctl, const long long *item_start)
{
    constexpr int g = batch_group_of(L);
    const int lane = threadIdx.x & 31;
    const int dry = ctl->dry;
    extern __shared__ unsigned long long sh_tq[];
    const TqBuf qb = warp_tq(sh_tq, SweepStyle<L>::TQ_LEN);
    const long long end = ctl->end[g];
    const int p0 = ctl->pbeg[g], p1 = ctl->pend[g];
    const BatchDesc *desc = ctl->desc;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(&ctl->next[g], 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= end) break;
        const BatchDesc d = desc[item_position(item_start, item, p0, p1)];
        batch_item_update<L>(d, item - d.item0, lane, dry, qb);
    }
}

template <int L>
static cudaError_t launch_b_sweep_t(BatchCtl *ctl, const long long *item_start, int grid, cudaStream_t s)
{
    constexpr size_t smem = tq_smem_bytes(SweepStyle<L>::TQ_LEN);
    static PerDeviceOnce once;
    cudaError_t e = once([] {
        return cudaFuncSetAttribute(k_b_sweep<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    k_b_sweep<L><<<grid, PA_BATCH_THREADS, smem, s>>>(ctl, item_start);
    return cudaGetLastError();
}

// One persistent launch for every run of the batch, whatever its lattice size: warps take
// items from one counter over all runs (in the order of k_b_items: by size, then by cost)
// and dispatch on the run's L to the same per-size item code.  Its tie queues are sized for
// the largest size's need.
constexpr int tq_len_max()
{
    int m = SweepStyle<4>::TQ_LEN;
    m = m > SweepStyle<8>::TQ_LEN ? m : SweepStyle<8>::TQ_LEN;
    m = m > SweepStyle<12>::TQ_LEN ? m : SweepStyle<12>::TQ_LEN;
    m = m > SweepStyle<16>::TQ_LEN ? m : SweepStyle<16>::TQ_LEN;
    m = m > SweepStyle<24>::TQ_LEN ? m : SweepStyle<24>::TQ_LEN;
    m = m > SweepStyle<32>::TQ_LEN ? m : SweepStyle<32>::TQ_LEN;
    m = m > SweepStyle<48>::TQ_LEN ? m : SweepStyle<48>::TQ_LEN;
    m = m > SweepStyle<64>::TQ_LEN ? m : SweepStyle<64>::TQ_LEN;
    m = m > SweepStyle<128>::TQ_LEN ? m : SweepStyle<128>::TQ_LEN;
    return m;
}

__global__ void __launch_bounds__(PA_BATCH_THREADS, PA_BATCH_MIN_BLOCKS) k_b_sweep_all(BatchCtl *ctl,
                                                                          const long long *item_start, int n)
{
    const int lane = threadIdx.x & 31;
    const int dry = ctl->dry;
    extern __shared__ unsigned long long sh_tq[];
    const TqBuf qb = warp_tq(sh_tq, tq_len_max());
    const long long end = ctl->total_items;
    const BatchDesc *desc = ctl->desc;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(&ctl->next_item, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= end) break;
        const BatchDesc d = desc[item_position(item_start, item, 0, n)];
        const long long it = item - d.item0;
        switch (d.L) {
            case 4: batch_item_update<4>(d, it, lane, dry, qb); break;
            case 8: batch_item_update<8>(d, it, lane, dry, qb); break;
            case 12: batch_item_update<12>(d, it, lane, dry, qb); break;
            case 16: batch_item_update<16>(d, it, lane, dry, qb); break;
            case 24: batch_item_update<24>(d, it, lane, dry, qb); break;
            case 32: batch_item_update<32>(d, it, lane, dry, qb); break;
            case 48: batch_item_update<48>(d, it, lane, dry, qb); break;
            case 64: batch_item_update<64>(d, it, lane, dry, qb); break;
            case 128: batch_item_update<128>(d, it, lane, dry, qb); break;
            default: break;
        }
    }
}

cudaError_t launch_batch_sweep(BatchCtl *ctl, const long long *item_start, const BatchSweepPlan &plan, cudaStream_t s)
{
    if (plan.unified) {
        constexpr size_t smem = tq_smem_bytes(tq_len_max());
        static PerDeviceOnce once;
        cudaError_t e = once([] {
            return cudaFuncSetAttribute(k_b_sweep_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        if (e != cudaSuccess) return e;
        k_b_sweep_all<<<plan.grid_all, PA_BATCH_THREADS, smem, s>>>(ctl, item_start, plan.n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // the runs without a register kernel (skipped above) by their own persistent sweep
        if (plan.any_present)
            e = launch_batch_sweep_any(ctl, item_start, plan.any_grid, plan.any_kw, s);
        return e;
    }
    cudaError_t e = cudaEventRecord(plan.fork, s);
    for (int i = 0; i < plan.ngroups && e == cudaSuccess; ++i) {
        cudaStream_t t = plan.side[i];
        if ((e = cudaStreamWaitEvent(t, plan.fork, 0)) != cudaSuccess) break;
        switch (plan.L[i]) {
            case 4: e = launch_b_sweep_t<4>(ctl, item_start, plan.grid[i], t); break;
            case 8: e = launch_b_sweep_t<8>(ctl, item_start, plan.grid[i], t); break;
            case 12: e = launch_b_sweep_t<12>(ctl, item_start, plan.grid[i], t); break;
            case 16: e = launch_b_sweep_t<16>(ctl, item_start, plan.grid[i], t); break;
            case 24: e = launch_b_sweep_t<24>(ctl, item_start, plan.grid[i], t); break;
            case 32: e = launch_b_sweep_t<32>(ctl, item_start, plan.grid[i], t); break;
            case 48: e = launch_b_sweep_t<48>(ctl, item_start, plan.grid[i], t); break;
            case 64: e = launch_b_sweep_t<64>(ctl, item_start, plan.grid[i], t); break;
            case 128: e = launch_b_sweep_t<128>(ctl, item_start, plan.grid[i], t); break;
            default:  // the group of every even L without a register kernel
                e = launch_batch_sweep_any(ctl, item_start, plan.grid[i], plan.any_kw, t);
                break;
        }
        if (e == cudaSuccess) e = cudaEventRecord(plan.join[i], t);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan.join[i], 0);
    }
    return e;
}

template <int L>
static int b_sweep_occupancy()
{
    constexpr size_t smem = tq_smem_bytes(SweepStyle<L>::TQ_LEN);
    int b = 0;
    if (cudaFuncSetAttribute(k_b_sweep<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_b_sweep<L>, PA_BATCH_THREADS, smem) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

int batch_sweep_max_blocks_per_sm(int L)
{
    if (L == 0) {  // the kernel over every size
        constexpr size_t smem = tq_smem_bytes(tq_len_max());
        int b = 0;
        if (cudaFuncSetAttribute(k_b_sweep_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_b_sweep_all, PA_BATCH_THREADS, smem) != cudaSuccess)
            return 1;
        return b > 0 ? b : 1;
    }
    switch (L) {
        case 4: return b_sweep_occupancy<4>();
        case 8: return b_sweep_occupancy<8>();
        case 12: return b_sweep_occupancy<12>();
        case 16: return b_sweep_occupancy<16>();
        case 24: return b_sweep_occupancy<24>();
        case 32: return b_sweep_occupancy<32>();
        case 48: return b_sweep_occupancy<48>();
        case 64: return b_sweep_occupancy<64>();
        case 128: return b_sweep_occupancy<128>();
        default: return 1;
    }
}

}  // namespace pa
