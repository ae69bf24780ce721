// pa_resample.cu -- step 2 (reweighting, resampling, replica copying) and step 4
// (observables, families, free energy) of population annealing (arXiv:2102.06611, Sec. II),
// plus the hash / export kernels used to check the population against an independent CPU
// implementation.
//
// Step 2 on the device, for the energies measured before resampling:
//   k_table   one block: level histogram h_k -> E_ref (lowest occupied level),
//             w_k = exp(-dbeta (E_k - E_ref)), S = sum of h_k w_k over the occupied k in
//             ascending order, in a fixed pairwise order (1024 consecutive chunks, each summed
//             from its first term, then a binary tree), ln Q_i = -dbeta E_ref + ln(S / R_{i-1})
//             (Eq. Q), tau_hat_k = R w_k / S (Eq. taus), floor(tau_hat_k) and the integer
//             threshold floor(frac(tau_hat_k) 2^32).  All binary64 arithmetic uses explicitly
//             rounded intrinsics; this file is also built with -fmad=false.
//   k_counts  one thread per parent: nearest-integer copies (Eq. resampling-factors) from one
//             Philox word, or Poisson copies; per-block sums.
//   k_scan    one block: exclusive prefix sum of the block sums, R_i, capacity check.
//   k_copy    per block: exclusive scan of its parents' copy numbers, then a group of lanes
//             per parent (as many as the replica has 16-byte vectors, up to a warp) copies
//             its packed spins to its r_j consecutive child slots with the level,
//             magnetisation and family id (tree order).
#include <climits>

#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Workspace plan_workspace(int L, long long capacity)
{
    Workspace w{};
    const size_t nlev = (size_t)L * L + 1;
    const long long nblk = (capacity + kCountBlockItems - 1) / kCountBlockItems;
    const size_t words = (size_t)L * ((L + 31) / 32);
    size_t off = 0;
    w.state = off;    off = align256(off + sizeof(DevState));
    w.hist = off;     off = align256(off + nlev * 4);
    w.fl = off;       off = align256(off + nlev * 4);
    w.thr = off;      off = align256(off + nlev * 4);
    w.tau = off;      off = align256(off + nlev * 8);
    w.w = off;        off = align256(off + nlev * 8);
    w.counts = off;   off = align256(off + (size_t)capacity * 4);
    w.blocksum = off; off = align256(off + (size_t)nblk * 8);
    w.fampart = off;  off = align256(off + (size_t)kFamBlocks * 2 * 8);
    w.obs = off;      off = align256(off + sizeof(pa_obs));
    w.hashes = off;   off = align256(off + (size_t)capacity * 8);
    w.stage = off;    off = align256(off + (size_t)kStageReplicas * words * 4);
    w.occ_k = off;    off = align256(off + nlev * 4);
    w.occ_h = off;    off = align256(off + nlev * 4);
    w.occ_w = off;    off = align256(off + nlev * 8);
    w.occ_t = off;    off = align256(off + nlev * 8);
    w.feat = off;     off = align256(off + 32 * 4 + 8);
    w.snap = off;     off = align256(off + (size_t)capacity * 4);
    w.ana_blk = off;  off = align256(off + (size_t)kMaxAnaBlocks * 4 * 8);
    w.ana_sizes = off; off = align256(off + ((size_t)capacity + 1) * 4);
    w.ana_out = off;  off = align256(off + sizeof(pa_analysis));
    w.wint = off;     off = align256(off + nlev * 8);
    w.cdf = off;      off = align256(off + (size_t)capacity * 8);
    w.search = off;   off = align256(off + sizeof(SearchState));
    w.hist_before = off; off = align256(off + (size_t)nlev * 4);
    w.total = off;
    w.nblk = nblk;
    return w;
}


// Thresholds of the run's spin update at beta: Metropolis floor(e^{-4 beta} 2^32),
// floor(e^{-8 beta} 2^32); heatbath T_3 = floor(2^32 / (1 + e^{4 beta})), T_4 likewise with 8 beta.
__device__ __forceinline__ void set_thresholds(DevState *st, double beta)
{
    const double y4 = __dmul_rn(4.0, beta), y8 = __dmul_rn(8.0, beta);
    if (st->update == PA_UPDATE_HEATBATH) {
        st->T4 = heatbath_threshold(y4);
        st->T8 = heatbath_threshold(y8);
    } else {
        st->T4 = metropolis_threshold(y4);
        st->T8 = metropolis_threshold(y8);
    }
}

// ------------------------------------------------------------------------------ setup
__global__ void k_setup(DevState *st, long long R, int *hist, int nlev, int update)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevState z{};
        *st = z;
        st->R_cur = R;
        st->R_prev = 0;
        st->update = update;
        set_thresholds(st, 0.0);
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nlev; k += gridDim.x * blockDim.x) hist[k] = 0;
}

__device__ __forceinline__ void zero_measure_body(DevState *st, int *hist, int nlev)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->sum_absM = 0;
        st->sum_M2 = 0;
        st->c0 = st->c00 = st->c1 = st->c11 = st->c01 = 0;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nlev; k += gridDim.x * blockDim.x) hist[k] = 0;
}

__global__ void k_zero_measure(DevState *st, int *hist, int nlev) { zero_measure_body(st, hist, nlev); }

__global__ void k_thresholds(DevState *st, double beta) { set_thresholds(st, beta); }

cudaError_t launch_zero_measure(DevState *st, int *hist, int N, cudaStream_t s)
{
    const int nlev = N + 1;
    k_zero_measure<<<(nlev + 1023) / 1024, 1024, 0, s>>>(st, hist, nlev);
    return cudaGetLastError();
}

cudaError_t launch_thresholds(DevState *st, double beta, cudaStream_t s)
{
    k_thresholds<<<1, 1, 0, s>>>(st, beta);
    return cudaGetLastError();
}

cudaError_t launch_setup(DevState *st, long long R, int *hist, int N, int update, cudaStream_t s)
{
    const int nlev = N + 1;
    k_setup<<<(nlev + 1023) / 1024, 1024, 0, s>>>(st, R, hist, nlev, update);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ k_table
constexpr int kTableThreads = 1024;
// k_table's dynamic shared memory per level: the compacted products h_k w_k (binary64) and
// the occupied levels' indices (int32)
constexpr size_t kTableSmemPerLevel = sizeof(double) + sizeof(int);

__device__ __forceinline__ void table_body(const ResampleArgs &a)
{
    extern __shared__ double sh_prod[];  // compacted h_k w_k, ascending k; then the levels k
    __shared__ int sh_kmin;
    __shared__ double sh_S;
    DevState *st = a.st;
    if (st->error) return;
    const int N = a.L * a.L;
    const int nlev = N + 1;
    const int tid = threadIdx.x;

    // lowest occupied level
    int kmin_local = INT_MAX;
    for (int k = tid; k < nlev; k += kTableThreads)
        if (a.hist[k] > 0) kmin_local = min(kmin_local, k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kmin_local = min(kmin_local, __shfl_xor_sync(0xffffffffu, kmin_local, o));
    if (tid == 0) sh_kmin = INT_MAX;
    __syncthreads();
    if ((tid & 31) == 0) atomicMin(&sh_kmin, kmin_local);
    __syncthreads();
    const int kmin = sh_kmin;
    if (kmin == INT_MAX) {
        if (tid == 0) set_error(st, PA_ERR_NUMERIC);
        return;
    }
    const double dbeta = __dsub_rn(a.beta_new, a.beta_prev);
    const int Eref = 4 * kmin - 2 * N;

    // each thread owns a contiguous chunk of levels; compact the occupied ones in order, then
    // spread their binary64 work over the threads (position i of the occupied list: thread
    // i mod 1024), since the occupied levels are few and adjacent
    int *sh_occ = reinterpret_cast<int *>(sh_prod + nlev);
    const int chunk = (nlev + kTableThreads - 1) / kTableThreads;
    const int k_lo = min(tid * chunk, nlev), k_hi = min(k_lo + chunk, nlev);
    int occ = 0;
    for (int k = k_lo; k < k_hi; ++k) occ += a.hist[k] > 0;
    int nocc;
    int pos = block_exclusive_scan<int, kTableThreads>(occ, &nocc);
    for (int k = k_lo; k < k_hi; ++k)
        if (a.hist[k] > 0) sh_occ[pos++] = k;
    __syncthreads();
    for (int i = tid; i < nocc; i += kTableThreads) {
        const int k = sh_occ[i];
        const int Ek = 4 * k - 2 * N;
        const double wk = det_exp(-__dmul_rn(dbeta, (double)(Ek - Eref)));
        a.w[k] = wk;
        sh_prod[i] = __dmul_rn((double)a.hist[k], wk);
    }
    __syncthreads();
    // S in the fixed pairwise order: the nocc products (ascending levels) in 1024 consecutive
    // chunks of ceil(nocc / 1024), thread t summing chunk t from its first term, then a binary
    // tree over the chunk sums
    {
        static_assert(kTableThreads == 1024, "one chunk of the pairwise sum per thread");
        __shared__ double sh_part[kTableThreads];
        const int c = (nocc + kTableThreads - 1) / kTableThreads;
        const int i0 = min(tid * c, nocc), i1 = min(i0 + c, nocc);
        double part = 0.0;
        for (int i = i0; i < i1; ++i) part = __dadd_rn(part, sh_prod[i]);
        sh_part[tid] = part;
        __syncthreads();
        for (int s = kTableThreads / 2; s > 0; s >>= 1) {
            if (tid < s) sh_part[tid] = __dadd_rn(sh_part[tid], sh_part[tid + s]);
            __syncthreads();
        }
        if (tid == 0) sh_S = sh_part[0];
    }
    __syncthreads();
    const double S = sh_S;
    const double Rt = (double)a.R_target;
    unsigned long long wt = 0, wb = 0;  // this thread's levels: sum h_k W_k, and over the shards before
    for (int i = tid; i < nocc; i += kTableThreads) {
        const int k = sh_occ[i];
        const int h = a.hist[k];
        const double wk = a.w[k];
        const double tau = __ddiv_rn(__dmul_rn(Rt, wk), S);
        const double f = floor(tau);
        a.tau[k] = tau;
        a.fl[k] = (int)f;
        a.thr[k] = (unsigned int)floor(__dmul_rn(__dsub_rn(tau, f), 4294967296.0));
        if (a.kind == PA_RESAMPLE_MULTINOMIAL) {
            const unsigned long long W = (unsigned long long)floor(__dmul_rn(wk, 4294967296.0));
            a.wint[k] = W;
            wt += (unsigned long long)h * W;
            if (a.sharded) wb += (unsigned long long)a.hist_before[k] * W;
        }
    }
    if (a.kind == PA_RESAMPLE_MULTINOMIAL && a.sharded) {
        // a shard's parents take the range [B, B + its own weight sum) of the whole population's
        // running weight sum, whose total is T (exact integers: every shard gets the same T)
        wt = block_sum<unsigned long long, kTableThreads>(wt);
        wb = block_sum<unsigned long long, kTableThreads>(wb);
        if (tid == 0) {
            st->mn_total = wt;
            st->mn_base = wb;
        }
    }
    if (tid == 0) {
        // R_{i-1}: the whole population's size (a shard's own parents are st->R_cur)
        const long long Rp = a.sharded ? st->R_glob : st->R_cur;
        const double lnQ = __dadd_rn(-__dmul_rn(dbeta, (double)Eref), log(__ddiv_rn(S, (double)Rp)));
        st->lnQ = lnQ;
        st->sum_lnQ = __dadd_rn(st->sum_lnQ, lnQ);
        st->sum_lnR = __dadd_rn(st->sum_lnR, log(__ddiv_rn((double)Rp, (double)a.R_target)));
        st->S = S;
        st->kmin = kmin;
        st->R_prev = st->R_cur;
        set_thresholds(st, a.beta_new);
        if (!(S > 0.0) || !isfinite(S)) set_error(st, PA_ERR_NUMERIC);
    }
}

__global__ void __launch_bounds__(kTableThreads) k_table(ResampleArgs a) { table_body(a); }

// ------------------------------------------------------------------------------ counts
// Poisson(lambda) by sequential inversion (Devroye 1986, Ch. X.3); lambda >= 32 is split
// into m = ceil(lambda / 32) independent draws of mean lambda / m.  Chunk c of parent j
// uses Philox(ctr = (j, c, POISSON << 28, i)); u = ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53.
__device__ long long poisson_draw(double lambda, unsigned int j, unsigned int step, unsigned int k0,
                                  unsigned int k1)
{
    if (!(lambda > 0.0)) return 0;
    long long m = 1;
    if (lambda >= 32.0) m = (long long)ceil(__ddiv_rn(lambda, 32.0));
    const double mu = __ddiv_rn(lambda, (double)m);
    const double p0 = det_exp(-mu);
    long long total = 0;
    for (long long c = 0; c < m; ++c) {
        const uint4 x = philox(make_uint4(j, (unsigned int)c, kStreamPoisson << 28, step), k0, k1);
        const double u = __dmul_rn(__dadd_rn(__dmul_rn((double)(x.x >> 5), 67108864.0), (double)(x.y >> 6)),
                                   1.0 / 9007199254740992.0);
        double p = p0, F = p0;
        long long k = 0;
        while (u >= F && k < 1000) {
            k = k + 1;
            p = __ddiv_rn(__dmul_rn(p, mu), (double)k);
            F = __dadd_rn(F, p);
        }
        total += k;
    }
    return total;
}

__device__ __forceinline__ void counts_body(const ResampleArgs &a)
{
    DevState *st = a.st;
    if (st->error) return;
    const long long Rp = st->R_prev;
    const long long base = (long long)blockIdx.x * kCountBlockItems;
    long long sum = 0;
#pragma unroll
    for (int it = 0; it < kCountItems; ++it) {
        const long long j = base + it * kCountThreads + threadIdx.x;
        if (j < Rp) {
            const int k = a.level_src[j];
            const unsigned int jg = (unsigned int)j + a.parent_base;  // global parent index
            long long r;
            if (a.kind == PA_RESAMPLE_NEAREST) {
                const uint4 x = philox(make_uint4(jg, 0u, kStreamResample << 28, a.step), a.k0, a.k1);
                r = (long long)a.fl[k] + (x.x <= a.thr[k] ? 1 : 0);
            } else {
                r = poisson_draw(a.tau[k], jg, a.step, a.k0, a.k1);
            }
            if (r > INT_MAX) r = INT_MAX;  // the capacity check rejects this population
            a.counts[j] = (int)r;
            sum += r;
        }
    }
    const long long t = block_sum<long long, kCountThreads>(sum);
    if (threadIdx.x == 0) a.blocksum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kCountThreads) k_counts(ResampleArgs a) { counts_body(a); }

// ------------------------------------------------------------------------------ multinomial
// Fixed-size multinomial resampling (Sec. II): R_target children pick parents with
// probabilities proportional to the integer weights W_j = floor(w_{k(j)} 2^32).
//   k_mn_wsum   per-block sums of W_j (blocks of kCountBlockItems parents)
//   k_mn_wscan  exclusive scan of the block sums, total T into DevState::mn_total
//   k_mn_cdf    C_j = W_0 + ... + W_j (exact uint64), counts zeroed
//   k_mn_draw   child c: X = Philox words 1:0, U = floor(X T / 2^64), parent = first j with
//               C_j > U (binary search), counts[j] += 1
//   k_mn_csum   per-block sums of the counts, for k_scan and k_copy
__device__ __forceinline__ void mn_wsum_body(const ResampleArgs &a)
{
    if (a.st->error) return;
    const long long Rp = a.st->R_prev;
    const long long base = (long long)blockIdx.x * kCountBlockItems;
    long long sum = 0;
#pragma unroll
    for (int it = 0; it < kCountItems; ++it) {
        const long long j = base + it * kCountThreads + threadIdx.x;
        if (j < Rp) sum += (long long)a.wint[a.level_src[j]];
    }
    const long long t = block_sum<long long, kCountThreads>(sum);
    if (threadIdx.x == 0) a.blocksum[blockIdx.x] = t;
}

__device__ __forceinline__ void mn_wscan_body(const ResampleArgs &a)
{
    DevState *st = a.st;
    if (st->error) return;
    const long long nb = (st->R_prev + kCountBlockItems - 1) / kCountBlockItems;
    // a shard's running sum starts at the weight of the shards before it (k_table set it and
    // the whole population's total)
    long long carry = a.sharded ? (long long)st->mn_base : 0;
    for (long long start = 0; start < nb; start += 1024) {
        const long long b = start + threadIdx.x;
        const long long v = b < nb ? a.blocksum[b] : 0;
        long long tot;
        const long long ex = block_exclusive_scan<long long, 1024>(v, &tot);
        if (b < nb) a.blocksum[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && !a.sharded) st->mn_total = (unsigned long long)carry;
}

__device__ __forceinline__ void mn_cdf_body(const ResampleArgs &a)
{
    if (a.st->error) return;
    const long long Rp = a.st->R_prev;
    const long long base = (long long)blockIdx.x * kCountBlockItems;
    // thread t owns parents base + 4t .. base + 4t + 3
    long long wv[kCountItems];
    long long local = 0;
#pragma unroll
    for (int it = 0; it < kCountItems; ++it) {
        const long long j = base + threadIdx.x * kCountItems + it;
        wv[it] = j < Rp ? (long long)a.wint[a.level_src[j]] : 0;
        local += wv[it];
    }
    long long tot;
    long long run = block_exclusive_scan<long long, kCountThreads>(local, &tot) + a.blocksum[blockIdx.x];
#pragma unroll
    for (int it = 0; it < kCountItems; ++it) {
        const long long j = base + threadIdx.x * kCountItems + it;
        run += wv[it];
        if (j < Rp) {
            a.cdf[j] = (unsigned long long)run;
            a.counts[j] = 0;
        }
    }
}

__device__ __forceinline__ void mn_draw_body(const ResampleArgs &a)
{
    const DevState *st = a.st;
    if (st->error) return;
    const long long Rp = st->R_prev;
    if (Rp < 1) return;
    const unsigned long long T = st->mn_total;
    // the range of the running weight sum held by these parents: [0, T) for a whole
    // population; a shard draws every child and keeps those that land on its parents
    const unsigned long long w_lo = a.sharded ? st->mn_base : 0ull, w_hi = a.cdf[Rp - 1];
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < a.R_target;
         c += (long long)gridDim.x * blockDim.x) {
        const uint4 x = philox(make_uint4((unsigned int)c, 0u, kStreamMultinomial << 28, a.step), a.k0, a.k1);
        const unsigned long long X = ((unsigned long long)x.y << 32) | x.x;
        const unsigned long long U = __umul64hi(X, T);
        if (U < w_lo || U >= w_hi) continue;
        long long lo = 0, hi = Rp - 1;  // first j with C_j > U
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (a.cdf[mid] > U) hi = mid;
            else lo = mid + 1;
        }
        atomicAdd(&a.counts[lo], 1);
    }
}

__device__ __forceinline__ void mn_csum_body(const ResampleArgs &a)
{
    if (a.st->error) return;
    const long long Rp = a.st->R_prev;
    const long long base = (long long)blockIdx.x * kCountBlockItems;
    long long sum = 0;
#pragma unroll
    for (int it = 0; it < kCountItems; ++it) {
        const long long j = base + it * kCountThreads + threadIdx.x;
        if (j < Rp) sum += a.counts[j];
    }
    const long long t = block_sum<long long, kCountThreads>(sum);
    if (threadIdx.x == 0) a.blocksum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kCountThreads) k_mn_wsum(ResampleArgs a) { mn_wsum_body(a); }
__global__ void __launch_bounds__(1024) k_mn_wscan(ResampleArgs a) { mn_wscan_body(a); }
__global__ void __launch_bounds__(kCountThreads) k_mn_cdf(ResampleArgs a) { mn_cdf_body(a); }
__global__ void __launch_bounds__(kCountThreads) k_mn_draw(ResampleArgs a) { mn_draw_body(a); }
__global__ void __launch_bounds__(kCountThreads) k_mn_csum(ResampleArgs a) { mn_csum_body(a); }

// ------------------------------------------------------------------------------ scan
constexpr int kScanThreads = 1024;

__device__ __forceinline__ void scan_body(const ResampleArgs &a)
{
    DevState *st = a.st;
    if (st->error) return;
    const long long Rp = st->R_prev;
    const long long nb = (Rp + kCountBlockItems - 1) / kCountBlockItems;
    long long carry = 0;
    for (long long start = 0; start < nb; start += kScanThreads) {
        const long long b = start + threadIdx.x;
        const long long v = b < nb ? a.blocksum[b] : 0;
        long long tot;
        const long long ex = block_exclusive_scan<long long, kScanThreads>(v, &tot);
        if (b < nb) a.blocksum[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (a.sharded) st->R_cur = carry;  // a shard's children: re-split before they are stored
        else if (carry > a.capacity) set_error(st, PA_ERR_CAPACITY);
        else if (carry == 0) set_error(st, PA_ERR_NUMERIC);
        else st->R_cur = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan(ResampleArgs a) { scan_body(a); }

// ------------------------------------------------------------------------------ copy
// Block `blk` of kCountBlockItems parents; with nsub > 1 several blocks share it, block `part`
// copying the children of parents [part, part + 1) x kCountBlockItems / nsub of it (each scans
// the whole block's copy numbers for its offsets), for more parallelism when there are few
// parent blocks (large replicas, small populations).
__device__ __forceinline__ void copy_body(const ResampleArgs &a, int chunks16, long long blk = blockIdx.x,
                                          int part = 0, int nsub = 1)
{
    __shared__ int sh_cnt[kCountBlockItems];
    __shared__ long long sh_off[kCountBlockItems];
    DevState *st = a.st;
    if (st->error) return;
    const long long Rp = st->R_prev;
    const long long base = blk * kCountBlockItems;
    if (base >= Rp) return;
    // thread t scans parents base + 4t .. base + 4t + 3
    int c[kCountItems];
    long long local = 0;
#pragma unroll
    for (int it = 0; it < kCountItems; ++it) {
        const long long j = base + threadIdx.x * kCountItems + it;
        c[it] = j < Rp ? a.counts[j] : 0;
        local += c[it];
    }
    long long tot;
    long long off = block_exclusive_scan<long long, kCountThreads>(local, &tot) + a.blocksum[blk];
#pragma unroll
    for (int it = 0; it < kCountItems; ++it) {
        sh_cnt[threadIdx.x * kCountItems + it] = c[it];
        sh_off[threadIdx.x * kCountItems + it] = off;
        off += c[it];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.spins_src);
    uint4 *dst = reinterpret_cast<uint4 *>(a.spins_dst);
    const int span = kCountBlockItems / nsub;
    const int p_lo = part * span;
    const int nloc = (int)min((long long)(p_lo + span), Rp - base);
    // children [k_lo, k_hi) of a parent whose children start at index o, written at o + k - shift
    const bool win = a.win_n > 0;
    const long long shift = win ? a.win_lo : 0;
    auto clip = [&](long long o, int cnt, int &k_lo, int &k_hi) {
        k_lo = 0;
        k_hi = cnt;
        if (win) {
            k_lo = (int)max(0LL, min((long long)cnt, a.win_lo - o));
            k_hi = (int)max((long long)k_lo, min((long long)cnt, a.win_lo + a.win_n - o));
        }
    };
    if (chunks16 >= 32) {
        // a warp per parent
        for (int p = p_lo + wid; p < nloc; p += kCountThreads / 32) {
            const int cnt = sh_cnt[p];
            if (cnt == 0) continue;
            const long long j = base + p;
            const long long o = sh_off[p];
            int k_lo, k_hi;
            clip(o, cnt, k_lo, k_hi);
            if (k_lo >= k_hi) continue;
            for (int ch = lane; ch < chunks16; ch += 32) {
                const uint4 v = src[(size_t)j * chunks16 + ch];
                for (int k = k_lo; k < k_hi; ++k) dst[(size_t)(o + k - shift) * chunks16 + ch] = v;
            }
            const int lv = a.level_src[j], mg = a.mag_src[j], fm = a.fam_src[j];
            for (int k = k_lo + lane; k < k_hi; k += 32) {
                a.level_dst[o + k - shift] = lv;
                a.mag_dst[o + k - shift] = mg;
                a.fam_dst[o + k - shift] = fm;
            }
        }
        return;
    }
    // small replicas: a group of 2^gs lanes (the smallest power of two >= the replica's
    // 16-byte vectors) per parent, 32 / 2^gs parents per warp at a time
    int gs = 0;
    while ((1 << gs) < chunks16) ++gs;
    const int S = 1 << gs, sub = lane >> gs, li = lane & (S - 1), per_warp = 32 >> gs;
    for (int p0 = p_lo + wid * per_warp; p0 < nloc; p0 += (kCountThreads / 32) * per_warp) {
        const int p = p0 + sub;
        if (p >= nloc) continue;
        const int cnt = sh_cnt[p];
        if (cnt == 0) continue;
        const long long j = base + p;
        const long long o = sh_off[p];
        int k_lo, k_hi;
        clip(o, cnt, k_lo, k_hi);
        if (k_lo >= k_hi) continue;
        if (li < chunks16) {
            const uint4 v = src[(size_t)j * chunks16 + li];
            for (int k = k_lo; k < k_hi; ++k) dst[(size_t)(o + k - shift) * chunks16 + li] = v;
        }
        const int lv = a.level_src[j], mg = a.mag_src[j], fm = a.fam_src[j];
        for (int k = k_lo + li; k < k_hi; k += S) {
            a.level_dst[o + k - shift] = lv;
            a.mag_dst[o + k - shift] = mg;
            a.fam_dst[o + k - shift] = fm;
        }
    }
}

__global__ void __launch_bounds__(kCountThreads) k_copy(ResampleArgs a, int chunks16, int nsub)
{
    copy_body(a, chunks16, blockIdx.x / nsub, (int)(blockIdx.x % nsub), nsub);
}

// Blocks sharing one block of parents: more when there are few parent blocks (up to ~8 blocks
// of 256 threads per SM of a 152-SM GPU).
static int copy_split(long long nblk) { return nblk <= 304 ? 4 : (nblk <= 608 ? 2 : 1); }

// k_table's dynamic shared-memory limit (up to 16385 doubles), raised once per device
static PerDeviceOnce table_smem_once;

cudaError_t launch_resample(const ResampleArgs &a, cudaStream_t s)
{
    const int nlev = a.L * a.L + 1;
    const size_t smem = (size_t)nlev * kTableSmemPerLevel;
    {
        cudaError_t e = table_smem_once([] {
            return cudaFuncSetAttribute(k_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((size_t)(128 * 128 + 1) * kTableSmemPerLevel));
        });
        if (e != cudaSuccess) return e;
    }
    k_table<<<1, kTableThreads, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned int nblk = (unsigned int)a.nblk;
    if (a.kind == PA_RESAMPLE_MULTINOMIAL) {
        k_mn_wsum<<<nblk, kCountThreads, 0, s>>>(a);
        k_mn_wscan<<<1, 1024, 0, s>>>(a);
        k_mn_cdf<<<nblk, kCountThreads, 0, s>>>(a);
        const long long dblk = (a.R_target + kCountThreads - 1) / kCountThreads;
        k_mn_draw<<<(unsigned int)(dblk < 4096 ? dblk : 4096), kCountThreads, 0, s>>>(a);
        k_mn_csum<<<nblk, kCountThreads, 0, s>>>(a);
    } else {
        k_counts<<<nblk, kCountThreads, 0, s>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_scan<<<1, kScanThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int chunks16 = bytes_per_replica(a.L) / 16;
    const int nsub = copy_split(a.nblk);
    k_copy<<<nblk * (unsigned int)nsub, kCountThreads, 0, s>>>(a, chunks16, nsub);
    return cudaGetLastError();
}

// The replica copy alone (children of the parents in spins_src ... into spins_dst ..., or the
// window [win_lo, win_lo + win_n) of them), after the copy numbers and their offsets.
cudaError_t launch_copy(const ResampleArgs &a, cudaStream_t s)
{
    const int chunks16 = bytes_per_replica(a.L) / 16;
    const int nsub = copy_split(a.nblk);
    k_copy<<<(unsigned int)a.nblk * (unsigned int)nsub, kCountThreads, 0, s>>>(a, chunks16, nsub);
    return cudaGetLastError();
}

// Level table, copy numbers and their total, without the replica copy (used by the
// no-workspace entry point, whose scratch is a static device array, and by shards).
cudaError_t launch_copy_numbers(const ResampleArgs &a, cudaStream_t s)
{
    const int nlev = a.L * a.L + 1;
    const size_t smem = (size_t)nlev * kTableSmemPerLevel;
    {
        cudaError_t e = table_smem_once([] {
            return cudaFuncSetAttribute(k_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((size_t)(128 * 128 + 1) * kTableSmemPerLevel));
        });
        if (e != cudaSuccess) return e;
    }
    k_table<<<1, kTableThreads, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned int nblk = (unsigned int)a.nblk;
    if (a.kind == PA_RESAMPLE_MULTINOMIAL) {
        k_mn_wsum<<<nblk, kCountThreads, 0, s>>>(a);
        k_mn_wscan<<<1, 1024, 0, s>>>(a);
        k_mn_cdf<<<nblk, kCountThreads, 0, s>>>(a);
        const long long dblk = (a.R_target + kCountThreads - 1) / kCountThreads;
        k_mn_draw<<<(unsigned int)(dblk < 4096 ? dblk : 4096), kCountThreads, 0, s>>>(a);
        k_mn_csum<<<nblk, kCountThreads, 0, s>>>(a);
    } else {
        k_counts<<<nblk, kCountThreads, 0, s>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_scan<<<1, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ step 4
__device__ __forceinline__ void families_body(const DevState *st, const int *fam, long long *part)
{
    const long long R = st->R_cur;
    long long cnt = 0, s2 = 0;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < R;
         j += (long long)gridDim.x * blockDim.x) {
        const int f = fam[j];
        if (j > 0 && fam[j - 1] == f) continue;
        // run start: gallop, then bisect, for the first index with a different id
        long long lo = j, stepw = 1;
        while (lo + stepw < R && fam[lo + stepw] == f) {
            lo += stepw;
            stepw <<= 1;
        }
        long long hi = min(lo + stepw, R);
        while (hi - lo > 1) {
            const long long mid = lo + (hi - lo) / 2;
            if (fam[mid] == f) lo = mid;
            else hi = mid;
        }
        const long long len = hi - j;
        cnt += 1;
        s2 += len * len;
    }
    const long long c = block_sum<long long, 256>(cnt);
    const long long t = block_sum<long long, 256>(s2);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = c;
        part[2 * blockIdx.x + 1] = t;
    }
}

__device__ __forceinline__ void obs_body(const ObsArgs &a)
{
    const DevState *st = a.st;
    const int N = a.L * a.L;
    long long sE = 0, sE2 = 0;
    for (int k = threadIdx.x; k <= N; k += 1024) {
        const long long h = a.hist[k];
        const long long E = 4LL * k - 2LL * N;
        sE += h * E;
        sE2 += h * E * E;
    }
    long long fc = 0, f2 = 0;
    for (int b = threadIdx.x; b < kFamBlocks; b += 1024) {
        fc += a.fampart[2 * b];
        f2 += a.fampart[2 * b + 1];
    }
    sE = block_sum<long long, 1024>(sE);
    sE2 = block_sum<long long, 1024>(sE2);
    fc = block_sum<long long, 1024>(fc);
    f2 = block_sum<long long, 1024>(f2);
    if (threadIdx.x != 0) return;
    if (a.glob) {  // sharded population: the combined whole-population values
        fc = st->fam_count;
        f2 = st->fam_size2;
    }
    const long long R = a.glob ? st->R_glob : st->R_cur;
    const double Rd = (double)R, Nd = (double)N, b = a.beta;
    const double meanE = __ddiv_rn((double)sE, Rd);
    const double meanE2 = __ddiv_rn((double)sE2, Rd);
    pa_obs o;
    o.step = a.step;
    o.R = R;
    o.beta = a.beta;
    o.dbeta = a.dbeta;
    o.e = __ddiv_rn(meanE, Nd);
    o.C = __ddiv_rn(__dmul_rn(__dmul_rn(b, b), __dsub_rn(meanE2, __dmul_rn(meanE, meanE))), Nd);
    o.m = __ddiv_rn(__ddiv_rn((double)st->sum_absM, Rd), Nd);
    o.m2 = __ddiv_rn(__ddiv_rn((double)st->sum_M2, Rd), __dmul_rn(Nd, Nd));
    o.chi = __dmul_rn(__dmul_rn(b, Nd), __dsub_rn(o.m2, __dmul_rn(o.m, o.m)));
    o.lnQ = st->lnQ;
    o.minus_betaF = __dadd_rn(__dmul_rn(Nd, 0.6931471805599453094), st->sum_lnQ);
    o.rho_t = __ddiv_rn((double)f2, Rd);
    o.families = fc;
    o.sum_E = sE;
    o.sum_E2 = sE2;
    o.sum_absM = (long long)st->sum_absM;
    o.sum_M2 = (long long)st->sum_M2;
    o.sum_size2 = f2;
    o.theta = a.theta;
    o.status = st->error;
    o.sum_lnRratio = st->sum_lnR;
    o.R_target = a.R_target;
    *a.dst = o;
}

__global__ void __launch_bounds__(256) k_families(const DevState *st, const int *fam, long long *part)
{
    families_body(st, fam, part);
}

__global__ void __launch_bounds__(1024) k_obs(ObsArgs a) { obs_body(a); }

cudaError_t launch_observables(const ObsArgs &a, cudaStream_t s)
{
    cudaError_t e;
    if (!a.glob) {
        k_families<<<kFamBlocks, 256, 0, s>>>(a.st, a.fam, a.fampart);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_obs<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_families(const DevState *st, const int *fam, long long *fampart, cudaStream_t s)
{
    k_families<<<kFamBlocks, 256, 0, s>>>(st, fam, fampart);
    return cudaGetLastError();
}


// ------------------------------------------------------------------------------ batches
// One temperature step of every active run: begin (advance beta_i = i / (n_temps - 1)),
// table, counts, scan, copy, flip (switch buffers, count sweep work items), zero, sweep
// (persistent, pa_sweep.cu), families, record.  Every argument is read from device memory,
// so the sequence is captured once in a CUDA graph and replayed per step.
__global__ void k_b_begin(const BatchRun *runs, BatchState *state, int n)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        BatchState &s = state[r];
        if (!s.active) continue;
        const int err = runs[r].rs[s.cur].st->error;
        if (err) {
            s.active = 0;
            s.status = err;
        } else if (s.step >= runs[r].n_temps - 1) {
            s.active = 0;
        } else {
            s.beta_prev = s.beta;
            s.step += 1;
            s.beta = __ddiv_rn((double)s.step, (double)(runs[r].n_temps - 1));
        }
    }
}

__device__ __forceinline__ ResampleArgs batch_resample_args(const BatchRun &run, const BatchState &s)
{
    ResampleArgs a = run.rs[s.cur];
    a.beta_prev = s.beta_prev;
    a.beta_new = s.beta;
    a.step = (unsigned int)s.step;
    return a;
}

__global__ void __launch_bounds__(kTableThreads) k_b_table(const BatchRun *runs, const BatchState *state)
{
    const BatchState s = state[blockIdx.y];
    if (!s.active) return;
    table_body(batch_resample_args(runs[blockIdx.y], s));
}

__global__ void __launch_bounds__(kCountThreads) k_b_counts(const BatchRun *runs, const BatchState *state)
{
    const BatchState s = state[blockIdx.y];
    if (!s.active || blockIdx.x >= runs[blockIdx.y].rs[0].nblk ||
        runs[blockIdx.y].rs[0].kind == PA_RESAMPLE_MULTINOMIAL)
        return;
    counts_body(batch_resample_args(runs[blockIdx.y], s));
}

// Multinomial resampling of the batch's multinomial runs (the single-run kernels' bodies).
__device__ __forceinline__ bool b_mn_run(const BatchRun *runs, const BatchState *state, bool per_block)
{
    const BatchState &s = state[blockIdx.y];
    return s.active && runs[blockIdx.y].rs[0].kind == PA_RESAMPLE_MULTINOMIAL &&
           (!per_block || blockIdx.x < runs[blockIdx.y].rs[0].nblk);
}

__global__ void __launch_bounds__(kCountThreads) k_b_mn_wsum(const BatchRun *runs, const BatchState *state)
{
    if (b_mn_run(runs, state, true)) mn_wsum_body(batch_resample_args(runs[blockIdx.y], state[blockIdx.y]));
}

__global__ void __launch_bounds__(1024) k_b_mn_wscan(const BatchRun *runs, const BatchState *state)
{
    if (b_mn_run(runs, state, false)) mn_wscan_body(batch_resample_args(runs[blockIdx.y], state[blockIdx.y]));
}

__global__ void __launch_bounds__(kCountThreads) k_b_mn_cdf(const BatchRun *runs, const BatchState *state)
{
    if (b_mn_run(runs, state, true)) mn_cdf_body(batch_resample_args(runs[blockIdx.y], state[blockIdx.y]));
}

__global__ void __launch_bounds__(kCountThreads) k_b_mn_draw(const BatchRun *runs, const BatchState *state)
{
    if (b_mn_run(runs, state, false)) mn_draw_body(batch_resample_args(runs[blockIdx.y], state[blockIdx.y]));
}

__global__ void __launch_bounds__(kCountThreads) k_b_mn_csum(const BatchRun *runs, const BatchState *state)
{
    if (b_mn_run(runs, state, true)) mn_csum_body(batch_resample_args(runs[blockIdx.y], state[blockIdx.y]));
}

__global__ void __launch_bounds__(kScanThreads) k_b_scan(const BatchRun *runs, const BatchState *state)
{
    const BatchState s = state[blockIdx.y];
    if (!s.active) return;
    scan_body(batch_resample_args(runs[blockIdx.y], s));
}

__global__ void __launch_bounds__(kCountThreads) k_b_copy(const BatchRun *runs, const BatchState *state)
{
    const BatchState s = state[blockIdx.y];
    if (!s.active || blockIdx.x >= runs[blockIdx.y].rs[0].nblk) return;
    copy_body(batch_resample_args(runs[blockIdx.y], s), runs[blockIdx.y].chunks16);
}

// Switch each resampled run to its new buffers (unless resampling failed) and lay out the
// persistent sweep's work items: ceil(R_i / replicas-per-item) per run, runs in `order`.
__global__ void __launch_bounds__(1024) k_b_items(const BatchRun *runs, BatchState *state, BatchCtl *ctl,
                                                  const int *order, long long *item_start, int n, int flip)
{
    // one thread per run position (chunks of 1024), work items per run, exclusive scan, and
    // the position's sweep descriptor
    long long carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int p = base + (int)threadIdx.x;
        long long items = 0, R = 0;
        if (p < n) {
            const int r = order[p];
            BatchState &s = state[r];
            if (s.active) {
                const DevState *dst = runs[r].rs[s.cur].st;
                if (!dst->error) {
                    if (flip) s.cur ^= 1;
                    R = dst->R_cur;
                    const long long per_item = (long long)runs[r].rpw * runs[r].ipw;
                    items = (R + per_item - 1) / per_item;
                }
            }
        }
        long long tot;
        const long long ex = block_exclusive_scan<long long, 1024>(items, &tot);
        if (p < n) {
            item_start[p] = carry + ex;
            const int r = order[p];
            const BatchState s = state[r];
            const BatchRun &run = runs[r];
            BatchDesc d;
            d.a = run.sw[s.cur];
            d.a.step = (unsigned int)s.step;
            d.a.t0 = 0;
            d.a.theta = run.theta;
            d.a.T4 = d.a.st->T4;
            d.a.T8 = d.a.st->T8;
            d.spare = run.sw[s.cur ^ 1].spins;
            d.item0 = carry + ex;
            d.R = R;
            d.ipw = run.ipw;
            d.L = run.L;
            ctl->desc[p] = d;
        }
        carry += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        item_start[n] = carry;
        ctl->total_items = carry;
        ctl->next_item = 0;
    }
    if (threadIdx.x < kBatchGroups) {
        const int g = threadIdx.x;
        const long long b0 = ctl->pbeg[g] < ctl->pend[g] ? item_start[ctl->pbeg[g]] : 0;
        const long long b1 = ctl->pbeg[g] < ctl->pend[g] ? (ctl->pend[g] == n ? carry : item_start[ctl->pend[g]]) : 0;
        ctl->begin[g] = b0;
        ctl->end[g] = b1;
        ctl->next[g] = (unsigned long long)b0;
    }
}

__global__ void __launch_bounds__(1024) k_b_zero(const BatchRun *runs, const BatchState *state)
{
    const BatchState s = state[blockIdx.y];
    if (!s.active) return;
    const SweepArgs &a = runs[blockIdx.y].sw[s.cur];
    const int L = runs[blockIdx.y].L;
    zero_measure_body(a.st, a.hist, L * L + 1);
}

__global__ void __launch_bounds__(256) k_b_families(const BatchRun *runs, const BatchState *state)
{
    const BatchState s = state[blockIdx.y];
    if (!s.active) return;  // a finished run keeps its last record
    const ObsArgs &a = runs[blockIdx.y].obs[s.cur];
    families_body(a.st, a.fam, a.fampart);
}

__global__ void __launch_bounds__(1024) k_b_obs(const BatchRun *runs, BatchState *state, pa_obs *records)
{
    const BatchState s = state[blockIdx.y];
    if (!s.active) return;  // a finished run keeps its last record
    ObsArgs a = runs[blockIdx.y].obs[s.cur];
    a.step = s.step;
    a.beta = s.beta;
    a.dbeta = s.step > 0 ? __dsub_rn(s.beta, s.beta_prev) : 0.0;
    a.theta = s.step > 0 ? runs[blockIdx.y].theta : 0;
    a.dst = records + blockIdx.y;
    obs_body(a);
    // the run is finished once its last temperature is recorded
    if (threadIdx.x == 0 && s.step >= runs[blockIdx.y].n_temps - 1) state[blockIdx.y].active = 0;
}

cudaError_t launch_batch_items(const BatchRun *runs, BatchState *state, BatchCtl *ctl, const int *order,
                               long long *item_start, int n, int flip, cudaStream_t s)
{
    k_b_items<<<1, 1024, 0, s>>>(runs, state, ctl, order, item_start, n, flip);
    return cudaGetLastError();
}

cudaError_t launch_batch_record(const BatchRun *runs, BatchState *state, pa_obs *records, int n,
                                cudaStream_t s)
{
    k_b_families<<<dim3(kFamBlocks, n), 256, 0, s>>>(runs, state);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_b_obs<<<dim3(1, n), 1024, 0, s>>>(runs, state, records);
    return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchRun *runs, BatchState *state, BatchCtl *ctl, const int *order,
                              long long *item_start, pa_obs *records, int n, int nblk_max, int nlev_max,
                              int mn_draw_blocks, const BatchSweepPlan &plan, cudaStream_t s)
{
    {
        static PerDeviceOnce once;
        cudaError_t e = once([] {
            return cudaFuncSetAttribute(k_b_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((size_t)(128 * 128 + 1) * kTableSmemPerLevel));
        });
        if (e != cudaSuccess) return e;
    }
    cudaError_t e;
    k_b_begin<<<1, 256, 0, s>>>(runs, state, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_b_table<<<dim3(1, n), kTableThreads, (size_t)nlev_max * kTableSmemPerLevel, s>>>(runs, state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_b_counts<<<dim3(nblk_max, n), kCountThreads, 0, s>>>(runs, state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (mn_draw_blocks > 0) {
        k_b_mn_wsum<<<dim3(nblk_max, n), kCountThreads, 0, s>>>(runs, state);
        k_b_mn_wscan<<<dim3(1, n), 1024, 0, s>>>(runs, state);
        k_b_mn_cdf<<<dim3(nblk_max, n), kCountThreads, 0, s>>>(runs, state);
        k_b_mn_draw<<<dim3(mn_draw_blocks, n), kCountThreads, 0, s>>>(runs, state);
        k_b_mn_csum<<<dim3(nblk_max, n), kCountThreads, 0, s>>>(runs, state);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_b_scan<<<dim3(1, n), kScanThreads, 0, s>>>(runs, state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_b_copy<<<dim3(nblk_max, n), kCountThreads, 0, s>>>(runs, state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_batch_items(runs, state, ctl, order, item_start, n, 1, s)) != cudaSuccess) return e;
    k_b_zero<<<dim3((nlev_max + 1023) / 1024, n), 1024, 0, s>>>(runs, state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_batch_sweep(ctl, item_start, plan, s)) != cudaSuccess) return e;
    return launch_batch_record(runs, state, records, n, s);
}

// ------------------------------------------------------------------------------ hashes
// Canonical packed row: 32 columns per word, bit b of word w = spin at column 32w + b.
// The even-column half supplies the even bits, the odd-column half the odd bits.
__device__ __forceinline__ unsigned int spread16(unsigned int x)
{
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

template <typename W>
__device__ __forceinline__ unsigned int canonical_word(W E, W O, int w)
{
    const unsigned int e = (unsigned int)(E >> (16 * w)) & 0xFFFFu;
    const unsigned int o = (unsigned int)(O >> (16 * w)) & 0xFFFFu;
    return spread16(e) | (spread16(o) << 1);
}

template <typename W>
__global__ void k_hashes(int L, const W *spins, long long R_host, const DevState *st, unsigned long long *out)
{
    const long long R = st ? st->R_cur : R_host;
    const int nw = (L + 31) / 32;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < R;
         j += (long long)gridDim.x * blockDim.x) {
        const W *rep = spins + (size_t)j * 2 * L;
        unsigned long long h = 0xcbf29ce484222325ull;
        for (int r = 0; r < L; ++r) {
            const W E = rep[2 * r], O = rep[2 * r + 1];
            for (int w = 0; w < nw; ++w) {
                const unsigned int v = canonical_word<W>(E, O, w);
                for (int byte = 0; byte < 4; ++byte) {
                    h ^= (unsigned long long)((v >> (8 * byte)) & 0xFFu);
                    h *= 0x100000001b3ull;
                }
            }
        }
        out[j] = h;
    }
}

template <typename W>
__global__ void k_export(int L, const W *spins, long long first, long long count, unsigned int *out)
{
    const int nw = (L + 31) / 32;
    const long long total = count * L;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long jj = t / L;
        const int r = (int)(t % L);
        const W *rep = spins + (size_t)(first + jj) * 2 * L;
        const W E = rep[2 * r], O = rep[2 * r + 1];
        for (int w = 0; w < nw; ++w) out[(size_t)t * nw + w] = canonical_word<W>(E, O, w);
    }
}

cudaError_t launch_hashes(int L, const void *spins, long long R, const DevState *st,
                          unsigned long long *out, cudaStream_t s)
{
    const unsigned int blocks = (unsigned int)min((R + 255) / 256 + 1, 4096LL);
    if (L / 2 > 32) k_hashes<unsigned long long><<<blocks, 256, 0, s>>>(L, (const unsigned long long *)spins, R, st, out);
    else k_hashes<unsigned int><<<blocks, 256, 0, s>>>(L, (const unsigned int *)spins, R, st, out);
    return cudaGetLastError();
}

cudaError_t launch_export(int L, const void *spins, long long first, long long count, unsigned int *out,
                          cudaStream_t s)
{
    const unsigned int blocks = (unsigned int)min((count * L + 255) / 256 + 1, 4096LL);
    if (L / 2 > 32) k_export<unsigned long long><<<blocks, 256, 0, s>>>(L, (const unsigned long long *)spins, first, count, out);
    else k_export<unsigned int><<<blocks, 256, 0, s>>>(L, (const unsigned int *)spins, first, count, out);
    return cudaGetLastError();
}

}  // namespace pa
