// pa_schedule.cu -- the adaptive temperature step (arXiv:2102.06611, Sec. II: the step is
// chosen so that consecutive energy distributions overlap enough; Sec. X advises an overlap
// above about 0.7), on the device.
//
// Overlap of the current energy distribution with its reweighting to beta + dbeta:
//   alpha(dbeta) = sum over occupied levels k of min(p_k, q_k),
//   p_k = h_k (1 / R),  t_k = h_k w_k,  w_k = exp(-dbeta (E_k - E_ref)),  q_k = t_k (1 / S),
//   S = sum t_k (the reciprocals formed once: binary64 division is slow on this GPU),
// with E_ref the lowest occupied level's energy.  Both sums run over the occupied levels in
// ascending order in a fixed pairwise order: the n terms are cut into 1024 consecutive chunks
// of c = ceil(n / 1024) terms, each chunk is summed from its first term, and the 1024 chunk
// sums are added as a binary tree (x_i += x_{i + s} for s = 512, 256, ..., 1).  One block of
// 1024 threads evaluates alpha at one step, thread j owning chunk j.
//
// The step is the largest dbeta in (0, hi], hi = min(dbeta_max, beta_final - beta), with
// alpha(dbeta) >= alpha_target: hi itself if it qualifies, else a search on [0, hi] that
// narrows the bracket [lo, hi) (alpha(lo) >= target, lo = 0 at first) by a factor K = 64 per
// round: the K - 1 points x_m = lo + (hi - lo) (m / K) are evaluated at once, one block each,
// m* is the length of the prefix of points that reach the target, and the new bracket is
// [x_{m*}, x_{m*+1}) (x_0 = lo, x_K = hi).  ceil(iters / 6) rounds narrow it by 2^-iters.
// If no point ever qualifies the step is the smallest one tried (the final hi).
//
// Launch sequence (no host synchronisation between them): k_search_prep (compaction of the
// occupied levels, the proposal check of the learned schedule, alpha at hi), then one
// k_search_round per round, then k_search_final.  Later launches do nothing once an earlier
// one has decided.
#include <climits>

#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {
namespace {

constexpr int kSearchThreads = 1024;
constexpr int kMaxChunk = (128 * 128 + 1 + kSearchThreads - 1) / kSearchThreads;  // 17

struct Levels {
    const int *k, *h;
    int n, N, Eref;
    double invR;  // 1 / R
};

// alpha(dbeta) for one block (all threads call; the result is valid in every thread).
__device__ double overlap_block(const Levels &lv, double dbeta, double *sh)
{
    const int tid = threadIdx.x;
    const int c = (lv.n + kSearchThreads - 1) / kSearchThreads;
    const int i0 = min(tid * c, lv.n), i1 = min(i0 + c, lv.n);
    double t[kMaxChunk];
    double part = 0.0;
    for (int i = i0; i < i1; ++i) {
        const int Ek = 4 * lv.k[i] - 2 * lv.N;
        const double w = det_exp(-__dmul_rn(dbeta, (double)(Ek - lv.Eref)));
        t[i - i0] = __dmul_rn((double)lv.h[i], w);
        part = __dadd_rn(part, t[i - i0]);
    }
    sh[tid] = part;
    __syncthreads();
    for (int s = kSearchThreads / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = __dadd_rn(sh[tid], sh[tid + s]);
        __syncthreads();
    }
    if (tid == 0) sh[0] = __ddiv_rn(1.0, sh[0]);  // 1 / S
    __syncthreads();
    const double invS = sh[0];
    __syncthreads();
    part = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double pk = __dmul_rn((double)lv.h[i], lv.invR);
        const double qk = __dmul_rn(t[i - i0], invS);
        part = __dadd_rn(part, pk < qk ? pk : qk);
    }
    sh[tid] = part;
    __syncthreads();
    for (int s = kSearchThreads / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = __dadd_rn(sh[tid], sh[tid + s]);
        __syncthreads();
    }
    const double alpha = sh[0];
    __syncthreads();
    return alpha;
}

__device__ __forceinline__ Levels levels_of(const BisectArgs &a, const SearchState *ss)
{
    return Levels{a.occ_k, a.occ_h, ss->nocc, a.L * a.L, 4 * ss->kmin - 2 * a.L * a.L, ss->invR};
}

// The bracket after a round: m* = length of the qualifying prefix of the K - 1 points.
__device__ __forceinline__ void refine(const SearchBracket &b, const double *alpha, double target, SearchBracket &out)
{
    const double d = __dsub_rn(b.hi, b.lo);
    int m = 0;
    while (m + 1 < kSearchK && alpha[m + 1] >= target) ++m;
    out = b;
    if (m > 0) {
        out.lo = __dadd_rn(b.lo, __dmul_rn(d, (double)m / (double)kSearchK));
        out.a_lo = alpha[m];
    }
    if (m + 1 < kSearchK) out.hi = __dadd_rn(b.lo, __dmul_rn(d, (double)(m + 1) / (double)kSearchK));
}

__global__ void __launch_bounds__(kSearchThreads) k_search_prep(BisectArgs a, SearchState *ss)
{
    __shared__ double sh[kSearchThreads];
    __shared__ int sh_nocc;
    __shared__ long long sh_R;
    const int N = a.L * a.L, nlev = N + 1, tid = threadIdx.x;
    DevState *st = a.st;

    // compact the occupied levels in ascending order
    const int chunk = (nlev + kSearchThreads - 1) / kSearchThreads;
    const int k_lo = min(tid * chunk, nlev), k_hi = min(k_lo + chunk, nlev);
    int occ = 0;
    long long rsum = 0;
    for (int k = k_lo; k < k_hi; ++k) {
        occ += a.hist[k] > 0;
        rsum += a.hist[k];
    }
    int nocc;
    int pos = block_exclusive_scan<int, kSearchThreads>(occ, &nocc);
    const long long R = block_sum<long long, kSearchThreads>(rsum);
    for (int k = k_lo; k < k_hi; ++k) {
        const int h = a.hist[k];
        if (h > 0) {
            a.occ_k[pos] = k;
            a.occ_h[pos] = h;
            ++pos;
        }
    }
    __shared__ double sh_invR;
    if (tid == 0) {
        sh_R = R;
        sh_invR = __ddiv_rn(1.0, (double)R);
    }
    __syncthreads();
    if (tid == 0) {
        ss->nocc = nocc;
        ss->R = sh_R;
        ss->invR = sh_invR;
        ss->kmin = nocc > 0 ? a.occ_k[0] : 0;
        sh_nocc = nocc;
    }
    __syncthreads();
    const Levels lv{a.occ_k, a.occ_h, sh_nocc, N, nocc > 0 ? 4 * a.occ_k[0] - 2 * N : 0, sh_invR};

    double hi = __dsub_rn(a.beta_final, a.beta);
    if (a.dbeta_max < hi) hi = a.dbeta_max;
    int done = 0, source = a.use_prop ? PA_SCHED_FALLBACK : PA_SCHED_BISECT;
    double dbeta = hi, alpha = 1.0;
    if (!(hi > 0.0) || nocc == 0) {
        done = 1;
        source = a.use_prop ? PA_SCHED_LEARNED : PA_SCHED_BISECT;
    } else {
        if (a.use_prop) {
            // a proposed step is kept if its overlap reaches the floor
            double dp = st->dbeta_prop;
            if (dp > hi) dp = hi;
            const double a_p = overlap_block(lv, dp, sh);
            if (a_p >= a.alpha_floor) {
                done = 1;
                dbeta = dp;
                alpha = a_p;
                source = PA_SCHED_LEARNED;
            }
        }
        if (!done) {
            const double a_hi = overlap_block(lv, hi, sh);
            if (a_hi >= a.alpha_target) {
                done = 1;
                dbeta = hi;
                alpha = a_hi;
            }
        }
    }
    if (tid == 0) {
        ss->done = done;
        ss->source = source;
        ss->hi0 = hi;
        ss->dbeta = dbeta;
        ss->alpha = alpha;
        SearchBracket b;
        b.lo = 0.0;
        b.hi = hi;
        b.a_lo = 1.0;
        ss->br[1] = b;  // read by round 0
    }
}

// Round r: bracket from round r - 1's points (or the prep's for r = 0), then block m (of
// K - 1) evaluates alpha at x_{m+1}.  Block 0 stores the bracket for round r + 1.
__global__ void __launch_bounds__(kSearchThreads) k_search_round(BisectArgs a, SearchState *ss, int r)
{
    __shared__ double sh[kSearchThreads];
    if (ss->done) return;
    SearchBracket b = ss->br[(r + 1) & 1];
    if (r > 0) {
        SearchBracket nb;
        refine(b, ss->alpha_pts[(r + 1) & 1], a.alpha_target, nb);
        b = nb;
    }
    const int m = blockIdx.x + 1;
    const double x = __dadd_rn(b.lo, __dmul_rn(__dsub_rn(b.hi, b.lo), (double)m / (double)kSearchK));
    const double al = overlap_block(levels_of(a, ss), x, sh);
    if (threadIdx.x == 0) {
        ss->alpha_pts[r & 1][m] = al;
        if (blockIdx.x == 0) ss->br[r & 1] = b;
    }
}

__global__ void __launch_bounds__(kSearchThreads) k_search_final(BisectArgs a, SearchState *ss, int rounds)
{
    __shared__ double sh[kSearchThreads];
    DevState *st = a.st;
    double dbeta = ss->dbeta, alpha = ss->alpha;
    if (!ss->done) {
        SearchBracket b;
        refine(ss->br[(rounds + 1) & 1], ss->alpha_pts[(rounds + 1) & 1], a.alpha_target, b);
        if (b.lo > 0.0) {
            dbeta = b.lo;
            alpha = b.a_lo;
        } else {  // no tried step reaches the target: take the smallest one tried
            dbeta = b.hi;
            alpha = overlap_block(levels_of(a, ss), b.hi, sh);
        }
    }
    if (threadIdx.x == 0) {
        const double hi0 = ss->hi0;
        const double beta_next = (ss->nocc == 0 || !(hi0 > 0.0) ||
                                  (dbeta == hi0 && hi0 == __dsub_rn(a.beta_final, a.beta)))
                                     ? a.beta_final
                                     : __dadd_rn(a.beta, dbeta);
        st->beta_next = beta_next;
        st->alpha_next = alpha;
        st->source_next = ss->source;
    }
}

}  // namespace

cudaError_t launch_bisect(const BisectArgs &a, SearchState *ss, cudaStream_t s)
{
    const int rounds = (a.iters + 5) / 6;  // 6 bits per round (K = 64)
    k_search_prep<<<1, kSearchThreads, 0, s>>>(a, ss);
    cudaError_t e = cudaGetLastError();
    for (int r = 0; r < rounds && e == cudaSuccess; ++r) {
        k_search_round<<<kSearchK - 1, kSearchThreads, 0, s>>>(a, ss, r);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    k_search_final<<<1, kSearchThreads, 0, s>>>(a, ss, rounds);
    return cudaGetLastError();
}

}  // namespace pa
