// pa_sweep_any.cu -- step 1 (simple-sampling initialisation) and step 3 (theta checkerboard
// sweeps, Metropolis or heatbath) of population annealing (arXiv:2102.06611, Sec. II) for
// any even lattice size 4 <= L <= 128 that has no kernel template of its own (the sizes
// 4, 8, 12, 16, 24, 32, 48, 64 and 128 run the register-resident kernels of pa_sweep.cuh).
//
// One warp owns one replica at a time and stages it in shared memory in its HBM layout
// (per row the even-column half-row word, then the odd-column one, bit p = column 2p or
// 2p + 1, here widened to 64 bits).  For one colour the lanes update rows lane, lane + 32,
// ... : a row's colour-q sites are its half (r + q) & 1, whose vertical neighbours are the
// same half of rows r -/+ 1 and whose horizontal neighbours are the other half of row r at
// positions p and p -/+ 1, all of the other colour, so the lanes of one colour never
// write what another lane reads.
//
// The random numbers and decisions are those of the register kernels, written for a
// run-time size: the uniform x of site p of row r, colour q, sweep t has its top 8 bits from
// 8 bit planes (bit n mod 32 of the words of Philox(ctr = (2 chunk + k / 4, slot,
// SWEEP << 28 | 2t + q, i)), n = r H' + p, chunk = n / 32, H' = the smallest power of two
// >= L / 2) and its low 24 bits from Philox(ctr = (64 r + p, slot, REFINE << 28 | 2t + q, i))
// word 0, drawn only when the top bits tie with the threshold.  A site with a aligned
// neighbours flips iff x < T_a: Metropolis (Sec. IV) T_0 = T_1 = T_2 = 2^32, T_3 =
// floor(e^{-4 beta} 2^32), T_4 = floor(e^{-8 beta} 2^32); heatbath T_a ~ 2^32 / (1 + e^{beta dE})
// with dE = 4a - 8, i.e. T_3, T_4 = floor(2^32 / (1 + e^{4 beta})), floor(2^32 / (1 +
// e^{8 beta})) from the host and T_1 = 2^32 - T_3, T_0 = 2^32 - T_4, T_2 = 2^31.  x < T_a is decided over a whole half-row at once by a borrow chain
// over the planes against each site's class threshold bits.
#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {
namespace {

using u64 = unsigned long long;

constexpr int kAnyWarps = 8;  // warps per block, one replica each at a time

// Class thresholds T_a, a = 0..4 aligned neighbours, split into top 8 and low 24 bits;
// always has bit a set iff T_a = 2^32 (every site of class a flips).
struct ClassThr {
    unsigned int top[5];
    unsigned int low[5];
    unsigned int always;
};

__device__ ClassThr class_thresholds(int update, u64 T4, u64 T8)
{
    const u64 two32 = 1ull << 32;
    u64 T[5];
    if (update == PA_UPDATE_HEATBATH) {
        T[0] = two32 - T8;
        T[1] = two32 - T4;
        T[2] = two32 >> 1;
    } else {
        T[0] = T[1] = T[2] = two32;
    }
    T[3] = T4;
    T[4] = T8;
    ClassThr c;
    c.always = 0;
    for (int a = 0; a < 5; ++a) {
        if (T[a] >= two32) {
            c.always |= 1u << a;
            c.top[a] = 0;
            c.low[a] = 0;
        } else {
            c.top[a] = (unsigned int)(T[a] >> 24);
            c.low[a] = (unsigned int)(T[a] & 0xFFFFFFull);
        }
    }
    return c;
}

// bit p <- bit p - 1 and bit p <- bit p + 1, periodic in H bits (m = the H-bit mask)
__device__ __forceinline__ u64 rot_from_below(u64 x, int H, u64 m) { return ((x << 1) | (x >> (H - 1))) & m; }
__device__ __forceinline__ u64 rot_from_above(u64 x, int H, u64 m) { return ((x >> 1) | (x << (H - 1))) & m; }

// The 8 bit planes of row r (bit p of plane k = bit 31 - k of site p's uniform).
__device__ void row_planes(int r, int HP, u64 m, unsigned int slot, unsigned int tag, unsigned int step,
                           unsigned int k0, unsigned int k1, u64 *pl)
{
    const unsigned int c2 = (kStreamSweep << 28) | tag;
    if (HP <= 32) {
        // the row's sites are bits off .. off + H - 1 of chunk n / 32, n = r H'
        const unsigned int n = (unsigned int)(r * HP);
        const unsigned int chunk = n >> 5, off = n & 31u;
        const uint4 a = philox(make_uint4(2 * chunk, slot, c2, step), k0, k1);
        const uint4 b = philox(make_uint4(2 * chunk + 1, slot, c2, step), k0, k1);
        const unsigned int w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        for (int k = 0; k < 8; ++k) pl[k] = (u64)(w[k] >> off) & m;
    } else {
        // H' = 64: sites 0..31 are chunk 2r, sites 32..63 chunk 2r + 1
        const unsigned int c0 = (unsigned int)(4 * r);
        const uint4 a0 = philox(make_uint4(c0, slot, c2, step), k0, k1);
        const uint4 a1 = philox(make_uint4(c0 + 1, slot, c2, step), k0, k1);
        const uint4 b0 = philox(make_uint4(c0 + 2, slot, c2, step), k0, k1);
        const uint4 b1 = philox(make_uint4(c0 + 3, slot, c2, step), k0, k1);
        const unsigned int lo[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const unsigned int hi[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        for (int k = 0; k < 8; ++k) pl[k] = ((u64)lo[k] | ((u64)hi[k] << 32)) & m;
    }
}

// One colour q of one sweep over the rows lane, lane + 32, ... of the warp's replica S
// (S[2r] = even-column half of row r, S[2r + 1] = odd-column half).
__device__ void half_sweep_any(u64 *S, int L, int q, unsigned int slot, unsigned int tag, unsigned int step,
                               unsigned int k0, unsigned int k1, const ClassThr &th, int lane)
{
    const int H = L / 2;
    int HP = 1;
    while (HP < H) HP *= 2;
    const u64 m = (H == 64) ? ~0ull : ((1ull << H) - 1ull);
    for (int r = lane; r < L; r += 32) {
        const int h = (r + q) & 1;  // the half holding colour q in row r
        const int ru = (r == 0) ? L - 1 : r - 1, rd = (r == L - 1) ? 0 : r + 1;
        const u64 s = S[2 * r + h];
        const u64 o = S[2 * r + (h ^ 1)];
        const u64 up = S[2 * ru + h], dn = S[2 * rd + h];
        // even-column sites (h = 0) see odd columns p - 1 and p; odd-column sites see p and p + 1
        const u64 side = h == 0 ? rot_from_below(o, H, m) : rot_from_above(o, H, m);
        // aligned-neighbour count a = x1 + x2 + x3 + x4 in three bit slices
        const u64 x1 = ~(s ^ up) & m, x2 = ~(s ^ dn) & m, x3 = ~(s ^ o) & m, x4 = ~(s ^ side) & m;
        const u64 s12 = x1 ^ x2, c12 = x1 & x2, s34 = x3 ^ x4, c34 = x3 & x4;
        const u64 b0 = s12 ^ s34, cr = s12 & s34;
        const u64 b1 = c12 ^ c34 ^ cr;
        const u64 b2 = (c12 & c34) | ((c12 ^ c34) & cr);
        u64 cls[5];
        cls[0] = ~b2 & ~b1 & ~b0 & m;
        cls[1] = ~b2 & ~b1 & b0 & m;
        cls[2] = ~b2 & b1 & ~b0 & m;
        cls[3] = ~b2 & b1 & b0 & m;
        cls[4] = b2 & m;
        u64 alw = 0;
        for (int a = 0; a < 5; ++a)
            if ((th.always >> a) & 1u) alw |= cls[a];

        u64 pl[8];
        row_planes(r, HP, m, slot, tag, step, k0, k1, pl);
        // borrow chain from the least significant plane: lt = x_top < T_top, eq = x_top == T_top
        u64 lt = 0, eq = m & ~alw;
        for (int k = 7; k >= 0; --k) {
            u64 tm = 0;  // bit 7 - k of each site's class threshold
            for (int a = 0; a < 5; ++a)
                if ((th.top[a] >> (7 - k)) & 1u) tm |= cls[a];
            const u64 np = ~pl[k];
            lt = (np & tm) | (np & lt) | (tm & lt);
            eq &= ~(pl[k] ^ tm);
        }
        u64 flip = alw | (lt & ~alw);
        // ties: the low 24 bits decide
        while (eq) {
            const int p = __ffsll((long long)eq) - 1;
            const u64 bit = 1ull << p;
            int a = 0;
            for (int c = 1; c < 5; ++c)
                if (cls[c] & bit) a = c;
            const uint4 x = philox(make_uint4((unsigned int)(64 * r + p), slot, (kStreamRefine << 28) | tag, step),
                                   k0, k1);
            if ((x.x & 0xFFFFFFu) < th.low[a]) flip |= bit;
            eq &= eq - 1ull;
        }
        S[2 * r + h] = s ^ flip;
    }
}

// Simple sampling (step 1): site n = r L + c takes bit n mod 32 of word n / 32 of the INIT
// stream, word w being lane w mod 4 of Philox(ctr = (w / 4, slot, INIT << 28, 0)).
__device__ void init_any(u64 *S, int L, unsigned int slot, unsigned int k0, unsigned int k1, int lane)
{
    for (int r = lane; r < L; r += 32) {
        u64 E = 0, O = 0;
        unsigned int cached = 0xffffffffu;
        uint4 x = make_uint4(0, 0, 0, 0);
        for (int c = 0; c < L; ++c) {
            const unsigned int n = (unsigned int)(r * L + c), w = n >> 5;
            if ((w >> 2) != cached) {
                cached = w >> 2;
                x = philox(make_uint4(cached, slot, kStreamInit << 28, 0u), k0, k1);
            }
            const unsigned int word = (w & 3) == 0 ? x.x : (w & 3) == 1 ? x.y : (w & 3) == 2 ? x.z : x.w;
            const u64 bit = (u64)((word >> (n & 31)) & 1u);
            if (c & 1) O |= bit << (c >> 1);
            else E |= bit << (c >> 1);
        }
        S[2 * r] = E;
        S[2 * r + 1] = O;
    }
}

template <bool INIT>
__global__ void __launch_bounds__(32 * kAnyWarps) k_sweep_any(SweepArgs a, int L)
{
    extern __shared__ u64 sh_dyn[];
    const int N = L * L, H = L / 2;
    u64 *S = sh_dyn + (threadIdx.x >> 5) * (2 * L);  // this warp's replica
    int *sh_hist = reinterpret_cast<int *>(sh_dyn + kAnyWarps * 2 * L);
    __shared__ unsigned long long sh_sum[7];
    for (int k = threadIdx.x; k <= N; k += blockDim.x) sh_hist[k] = 0;
    if (threadIdx.x < 7) sh_sum[threadIdx.x] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const long long R = INIT ? a.R_init : a.st->R_cur;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const ClassThr th = class_thresholds(a.update, a.T4, a.T8);
    if (!INIT && blockIdx.x == 0 && threadIdx.x == 0 && (a.T4 != a.st->T4 || a.T8 != a.st->T8))
        set_error(a.st, PA_ERR_NUMERIC);  // host and device thresholds disagree (never expected)
    const bool wide = H > 32;
    const u64 m = (H == 64) ? ~0ull : ((1ull << H) - 1ull);

    for (long long j = warp; j < R; j += nwarps) {
        if (INIT) {
            init_any(S, L, (unsigned int)j, a.k0, a.k1, lane);
        } else if (wide) {
            const u64 *src = reinterpret_cast<const u64 *>(a.spins) + (size_t)j * (2 * L);
            for (int w = lane; w < 2 * L; w += 32) S[w] = src[w];
        } else {
            const unsigned int *src = reinterpret_cast<const unsigned int *>(a.spins) + (size_t)j * (2 * L);
            for (int w = lane; w < 2 * L; w += 32) S[w] = src[w];
        }
        __syncwarp();
        for (int t = 0; t < a.theta; ++t)
            for (int q = 0; q < 2; ++q) {
                half_sweep_any(S, L, q, (unsigned int)j, (unsigned int)(2 * (a.t0 + t) + q), a.step, a.k0, a.k1, th,
                               lane);
                __syncwarp();
            }
        // measurement: antiparallel bonds (row r: (2p, 2p+1), (2p+1, 2p+2); column: r, r+1)
        int anti = 0, ups = 0;
        for (int r = lane; r < L; r += 32) {
            const int rn = (r == L - 1) ? 0 : r + 1;
            const u64 E = S[2 * r], O = S[2 * r + 1];
            anti += __popcll(E ^ O) + __popcll(O ^ rot_from_above(E, H, m)) + __popcll(E ^ S[2 * rn]) +
                    __popcll(O ^ S[2 * rn + 1]);
            ups += __popcll(E) + __popcll(O);
        }
        anti = group_sum<32>(anti);
        ups = group_sum<32>(ups);
        if (INIT || a.theta > 0) {
            if (wide) {
                u64 *dst = reinterpret_cast<u64 *>(a.spins) + (size_t)j * (2 * L);
                for (int w = lane; w < 2 * L; w += 32) dst[w] = S[w];
            } else {
                unsigned int *dst = reinterpret_cast<unsigned int *>(a.spins) + (size_t)j * (2 * L);
                for (int w = lane; w < 2 * L; w += 32) dst[w] = (unsigned int)S[w];
            }
        }
        __syncwarp();  // the stores have read S before the next replica overwrites it
        if (lane == 0) {
            const int level = anti >> 1;
            const int M = 2 * ups - N;
            unsigned long long v[7] = {(unsigned long long)(M < 0 ? -M : M), (unsigned long long)((long long)M * M),
                                       0, 0, 0, 0, 0};
            if (!INIT) {
                const unsigned long long k0 = (unsigned long long)(a.t0 == 0 ? a.level[j] : a.level_snap[j]);
                const unsigned long long k1 = (unsigned long long)level;
                if (a.t0 == 0) a.level_snap[j] = (int)k0;
                v[2] = k0;
                v[3] = k0 * k0;
                v[4] = k1;
                v[5] = k1 * k1;
                v[6] = k0 * k1;
            }
            a.level[j] = level;
            a.mag[j] = M;
            if (INIT) a.fam[j] = (int)j;
            atomicAdd(&sh_hist[level], 1);
            for (int i = 0; i < (INIT ? 2 : 7); ++i) atomicAdd(&sh_sum[i], v[i]);
        }
    }

    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&a.st->sum_absM, sh_sum[0]);
        atomicAdd(&a.st->sum_M2, sh_sum[1]);
        if (!INIT) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c0), sh_sum[2]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c00), sh_sum[3]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c1), sh_sum[4]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c11), sh_sum[5]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c01), sh_sum[6]);
        }
    }
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
        const int v = sh_hist[k];
        if (v) atomicAdd(&a.hist[k], v);
    }
}

// shared memory of a block: the replicas of its warps, then the level histogram
size_t any_smem_bytes(int L) { return (size_t)kAnyWarps * 2 * L * sizeof(u64) + (size_t)(L * L + 1) * sizeof(int); }

template <bool INIT>
cudaError_t launch_any_t(int L, const SweepArgs &a, int num_sms, cudaStream_t s)
{
    const size_t smem = any_smem_bytes(L);
    static bool attr_set = false;  // the limit is set once, for the largest L
    cudaError_t e = cudaSuccess;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_sweep_any<INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)any_smem_bytes(128));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_any<INIT>, 32 * kAnyWarps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long blocks = (a.R_bound + kAnyWarps - 1) / kAnyWarps;
    const long long cap = (long long)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_sweep_any<INIT><<<(unsigned int)blocks, 32 * kAnyWarps, smem, s>>>(a, L);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_any(int L, bool init, const SweepArgs &a, int num_sms, cudaStream_t s)
{
    if (L < 4 || L > 128 || (L & 1)) return cudaErrorInvalidValue;
    return init ? launch_any_t<true>(L, a, num_sms, s) : launch_any_t<false>(L, a, num_sms, s);
}

}  // namespace pa
