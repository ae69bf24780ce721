// pa_sweep_any.cu -- step 1 (simple-sampling initialisation) and step 3 (theta checkerboard
// sweeps, Metropolis or heatbath) of population annealing (arXiv:2102.06611, Sec. II) for
// any even lattice size 4 <= L <= 128 that has no kernel template of its own (the sizes
// 4, 8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96 and 128 run the register-resident kernels of
// pa_sweep.cuh; batches run the others through the batched form below).
//
// A warp stages its replicas in shared memory in their HBM layout (per row the even-column
// half-row word, then the odd-column one, bit p = column 2p or 2p + 1, widened to 64 bits).
// A row's colour-q sites are its half (r + q) & 1, whose vertical neighbours are the same
// half of rows r -/+ 1 and whose horizontal neighbours are the other half of row r at
// positions p and p -/+ 1, all of the other colour, so the lanes updating one colour never
// write what another lane reads.  For L <= 64 a lane updates one 32-site random-number chunk
// at a time (the P rows of the chunk packed into one word); for L > 64 one row (two chunks).
//
// The random numbers and decisions are those of the register kernels, written for a
// run-time size: the uniform x of site p of row r, colour q, sweep t has its top 8 bits from
// 8 bit planes (bit n mod 32 of the words of Philox(ctr = (2 chunk + k / 4, slot,
// SWEEP << 28 | 2t + q, i)), n = r H' + p, chunk = n / 32, H' = the smallest power of two
// >= L / 2) and its low 24 bits from Philox(ctr = (64 r + p, slot, REFINE << 28 | 2t + q, i))
// word 0, drawn only when the top bits tie with the threshold.  A site with a aligned
// neighbours flips iff x < T_a.  Metropolis (Sec. IV): T_0 = T_1 = T_2 = 2^32,
// T_3 = floor(e^{-4 beta} 2^32), T_4 = floor(e^{-8 beta} 2^32).  Heatbath: T_a ~ 2^32 /
// (1 + e^{beta dE}) with dE = 4a - 8, i.e. T_3 = floor(2^32 / (1 + e^{4 beta})) and
// T_4 = floor(2^32 / (1 + e^{8 beta})) from the host, T_1 = 2^32 - T_3, T_0 = 2^32 - T_4,
// T_2 = 2^31.  x < T_a is decided over a whole word at once by a borrow chain over the
// planes against each site's class threshold bits.
#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {
namespace {

using u64 = unsigned long long;

// Block shape (build knobs): PA_ANY_WARPS warps per block, at least PA_ANY_MIN_BLOCKS
// resident blocks per SM.  16 warps (so at most 128 registers) was measured best: 20-35 %
// faster than 8 warps with the registers unbounded (which the compiler then took above 128,
// halving the resident warps) and 3-7 % faster than 8 warps in two blocks per SM, except at
// L = 6 (-6 %).
#ifndef PA_ANY_WARPS
#define PA_ANY_WARPS 16
#endif
#ifndef PA_ANY_MIN_BLOCKS
#define PA_ANY_MIN_BLOCKS 1
#endif
constexpr int kAnyWarps = PA_ANY_WARPS;  // warps per block

// Class thresholds T_a, a = 0..4 aligned neighbours, split into top 8 and low 24 bits;
// always has bit a set iff T_a = 2^32 (every site of class a flips).  Metropolis only needs
// T_3 and T_4: the threshold bit of plane k is then all4 * sel[k] + m3[k] (m3[k] = all ones
// iff bit 7 - k of T_3's top bits is set; sel[k] = +1 / -1 / 0 where only T_4's, only T_3's
// or both or neither bits are set), one multiply-add instead of a test per class.
struct ClassThr {
    unsigned int top[5];
    unsigned int low[5];
    unsigned int always;
    int metropolis;
    unsigned int m3[8], sel[8];
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
    c.metropolis = update != PA_UPDATE_HEATBATH;
    for (int k = 0; k < 8; ++k) {
        const unsigned int b3 = (c.top[3] >> (7 - k)) & 1u, b4 = (c.top[4] >> (7 - k)) & 1u;
        c.m3[k] = b3 ? 0xFFFFFFFFu : 0u;
        c.sel[k] = (b3 == b4) ? 0u : (b4 ? 1u : 0xFFFFFFFFu);
    }
    return c;
}

// Geometry of a run-time size.  Narrow sizes (H' <= 32, L <= 64): the P = 32 / H' rows of
// one chunk are packed into one 32-bit word (field i = bits i H' .. i H' + H - 1 = row cP + i),
// so a chunk's two Philox calls serve all its rows; nch chunks per colour, Gc lanes per
// replica and k = 32 / Gc replicas per warp.  Wide sizes (L > 64): a row is two chunks, one
// 64-bit word; a lane takes rows, one replica per warp.
struct AnyGeo {
    int L, H, HP, P, nch, Gc, k;
    bool wide;
    u64 hmask;
};

__host__ __device__ AnyGeo any_geo(int L)
{
    AnyGeo g;
    g.L = L;
    g.H = L / 2;
    g.HP = 1;
    while (g.HP < g.H) g.HP *= 2;
    g.wide = g.HP > 32;
    g.hmask = (g.H == 64) ? ~0ull : ((1ull << g.H) - 1ull);
    if (g.wide) {
        g.P = 1;
        g.nch = L;
        g.Gc = 32;
    } else {
        g.P = 32 / g.HP;
        g.nch = (L + g.P - 1) / g.P;
        int n = 1;
        while (n < g.nch && n < 32) n *= 2;
        g.Gc = n;
    }
    g.k = 32 / g.Gc;
    return g;
}

// all4 * sel + m3 on each 32-bit half (all4, the sites whose four neighbours align)
template <typename W>
__device__ __forceinline__ W metropolis_bits(W all4, unsigned int sel, unsigned int m3)
{
    if constexpr (sizeof(W) == 4) {
        return all4 * sel + m3;
    } else {
        const unsigned int lo = (unsigned int)all4 * sel + m3, hi = (unsigned int)(all4 >> 32) * sel + m3;
        return ((W)hi << 32) | (W)lo;
    }
}

// Classes and the top-8-bit decision of one word: returns the decided flips; eq = the
// sites whose top bits tie with their class threshold, cls = the class masks (a aligned
// neighbours, a = 0..4; Metropolis: only classes 3 and 4, the others always flip).  Sites
// outside V stay clear.
template <typename W>
__device__ __forceinline__ W decide(W s, W up, W dn, W o, W side, W V, const W *pl, const ClassThr &th, W &eq,
                                    W *cls)
{
    const W x1 = ~(s ^ up) & V, x2 = ~(s ^ dn) & V, x3 = ~(s ^ o) & V, x4 = ~(s ^ side) & V;
    if (th.metropolis) {
        // a >= 3: both of one pair aligned and at least one of the other
        const W t12 = x1 & x2, t34 = x3 & x4;
        const W all4 = t12 & t34;
        const W ge3 = (t12 & (x3 | x4)) | (t34 & (x1 | x2));
        const W eq3 = ge3 & ~all4;
        cls[0] = cls[1] = cls[2] = 0;
        cls[3] = eq3;
        cls[4] = all4;
        W alw = V & ~ge3;
        if (th.always & 8u) alw |= eq3;
        if (th.always & 16u) alw |= all4;
        W lt = 0, e = V & ~alw;
        for (int k = 7; k >= 0; --k) {
            const W tm = metropolis_bits<W>(all4, th.sel[k], th.m3[k]);
            const W np = ~pl[k];
            lt = (np & tm) | (np & lt) | (tm & lt);
            e &= ~(pl[k] ^ tm);
        }
        eq = e;
        return alw | (lt & ~alw & V);  // tm has bits outside V where m3 is all ones
    }
    // aligned-neighbour count a = x1 + x2 + x3 + x4 in three bit slices
    const W s12 = x1 ^ x2, c12 = x1 & x2, s34 = x3 ^ x4, c34 = x3 & x4;
    const W b0 = s12 ^ s34, cr = s12 & s34;
    const W b1 = c12 ^ c34 ^ cr;
    const W b2 = (c12 & c34) | ((c12 ^ c34) & cr);
    cls[0] = ~b2 & ~b1 & ~b0 & V;
    cls[1] = ~b2 & ~b1 & b0 & V;
    cls[2] = ~b2 & b1 & ~b0 & V;
    cls[3] = ~b2 & b1 & b0 & V;
    cls[4] = b2 & V;
    W alw = 0;
    for (int a = 0; a < 5; ++a)
        if ((th.always >> a) & 1u) alw |= cls[a];
    // borrow chain from the least significant plane: lt = x_top < T_top, e = x_top == T_top
    W lt = 0, e = V & ~alw;
    for (int k = 7; k >= 0; --k) {
        W tm = 0;  // bit 7 - k of each site's class threshold
        for (int a = 0; a < 5; ++a)
            if ((th.top[a] >> (7 - k)) & 1u) tm |= cls[a];
        const W np = ~pl[k];
        lt = (np & tm) | (np & lt) | (tm & lt);
        e &= ~(pl[k] ^ tm);
    }
    eq = e;
    return alw | (lt & ~alw);
}

// The low 24 bits decide a tie: site p of row r, class a.
__device__ __forceinline__ bool tie_accept(int r, int p, int a, unsigned int slot, unsigned int tag, unsigned int step,
                                           unsigned int k0, unsigned int k1, const ClassThr &th)
{
    const uint4 x = philox(make_uint4((unsigned int)(64 * r + p), slot, (kStreamRefine << 28) | tag, step), k0, k1);
    // select with constant indices (a run-time index would move the thresholds to local memory)
    unsigned int low = th.low[0];
#pragma unroll
    for (int c = 1; c < 5; ++c)
        if (a == c) low = th.low[c];
    return (x.x & 0xFFFFFFu) < low;
}

template <typename W>
__device__ __forceinline__ int class_of(const W *cls, W bit)
{
    int a = 0;
    for (int c = 1; c < 5; ++c)
        if (cls[c] & bit) a = c;
    return a;
}

// One colour q of one sweep, narrow sizes: the lane updates chunks c0, c0 + Gc, ... of the
// replica S (S[2r] = even-column half of row r, S[2r + 1] = odd-column half).
__device__ __forceinline__ void half_sweep_chunks(u64 *S, const AnyGeo &g, int q, unsigned int slot, unsigned int tag,
                                  unsigned int step, unsigned int k0, unsigned int k1, const ClassThr &th, int c0)
{
    const int L = g.L, H = g.H, HP = g.HP, P = g.P;
    const unsigned int hm = (unsigned int)g.hmask;
    const unsigned int c2 = (kStreamSweep << 28) | tag;
    for (int c = c0; c < g.nch; c += g.Gc) {
        // pack the chunk's rows: T = colour-q sites, O = the other half of the same rows,
        // U / D = the same half of the rows above / below, Sd = O shifted to the second
        // horizontal neighbour (even-column sites see p - 1, odd-column sites p + 1)
        unsigned int T = 0, O = 0, U = 0, D = 0, Sd = 0, V = 0;
        for (int i = 0; i < P; ++i) {
            const int r = c * P + i;
            if (r >= L) break;
            const int h = (r + q) & 1;
            const int ru = (r == 0) ? L - 1 : r - 1, rd = (r == L - 1) ? 0 : r + 1;
            const unsigned int o = (unsigned int)S[2 * r + (h ^ 1)];
            const int sh = i * HP;
            T |= (unsigned int)S[2 * r + h] << sh;
            O |= o << sh;
            U |= (unsigned int)S[2 * ru + h] << sh;
            D |= (unsigned int)S[2 * rd + h] << sh;
            const unsigned int side = h == 0 ? ((o << 1) | (o >> (H - 1))) & hm : ((o >> 1) | (o << (H - 1))) & hm;
            Sd |= side << sh;
            V |= hm << sh;
        }
        // the chunk's 8 bit planes: bit n mod 32 = bit i H' + p
        const uint4 a0 = philox(make_uint4(2 * (unsigned int)c, slot, c2, step), k0, k1);
        const uint4 a1 = philox(make_uint4(2 * (unsigned int)c + 1, slot, c2, step), k0, k1);
        const unsigned int pl[8] = {a0.x & V, a0.y & V, a0.z & V, a0.w & V, a1.x & V, a1.y & V, a1.z & V, a1.w & V};
        unsigned int eq, cls[5];
        unsigned int flip = decide<unsigned int>(T, U, D, O, Sd, V, pl, th, eq, cls);
        while (eq) {
            const int b = __ffs((int)eq) - 1;
            const unsigned int bit = 1u << b;
            if (tie_accept(c * P + b / HP, b % HP, class_of(cls, bit), slot, tag, step, k0, k1, th)) flip |= bit;
            eq &= eq - 1u;
        }
        const unsigned int Tn = T ^ flip;
        for (int i = 0; i < P; ++i) {
            const int r = c * P + i;
            if (r >= L) break;
            S[2 * r + ((r + q) & 1)] = (Tn >> (i * HP)) & hm;
        }
    }
}

// One colour q of one sweep, wide sizes: the lane updates rows c0, c0 + 32, ... (one row =
// chunks 2r and 2r + 1, four Philox calls for its planes).
__device__ __forceinline__ void half_sweep_rows(u64 *S, const AnyGeo &g, int q, unsigned int slot, unsigned int tag,
                                unsigned int step, unsigned int k0, unsigned int k1, const ClassThr &th, int c0)
{
    const int L = g.L, H = g.H;
    const u64 m = g.hmask;
    const unsigned int c2 = (kStreamSweep << 28) | tag;
    for (int r = c0; r < L; r += g.Gc) {
        const int h = (r + q) & 1;  // the half holding colour q in row r
        const int ru = (r == 0) ? L - 1 : r - 1, rd = (r == L - 1) ? 0 : r + 1;
        const u64 s = S[2 * r + h];
        const u64 o = S[2 * r + (h ^ 1)];
        const u64 side = h == 0 ? ((o << 1) | (o >> (H - 1))) & m : ((o >> 1) | (o << (H - 1))) & m;
        const unsigned int ch = (unsigned int)(4 * r);
        const uint4 a0 = philox(make_uint4(ch, slot, c2, step), k0, k1);
        const uint4 a1 = philox(make_uint4(ch + 1, slot, c2, step), k0, k1);
        const uint4 b0 = philox(make_uint4(ch + 2, slot, c2, step), k0, k1);
        const uint4 b1 = philox(make_uint4(ch + 3, slot, c2, step), k0, k1);
        const unsigned int lo[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const unsigned int hi[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        u64 pl[8];
        for (int k = 0; k < 8; ++k) pl[k] = ((u64)lo[k] | ((u64)hi[k] << 32)) & m;
        u64 eq, cls[5];
        u64 flip = decide<u64>(s, S[2 * ru + h], S[2 * rd + h], o, side, m, pl, th, eq, cls);
        while (eq) {
            const int p = __ffsll((long long)eq) - 1;
            const u64 bit = 1ull << p;
            if (tie_accept(r, p, class_of(cls, bit), slot, tag, step, k0, k1, th)) flip |= bit;
            eq &= eq - 1ull;
        }
        S[2 * r + h] = s ^ flip;
    }
}

// Simple sampling (step 1): site n = r L + c takes bit n mod 32 of word n / 32 of the INIT
// stream, word w being lane w mod 4 of Philox(ctr = (w / 4, slot, INIT << 28, 0)).  The lane
// fills rows c0, c0 + Gc, ...
__device__ void init_any(u64 *S, const AnyGeo &g, unsigned int slot, unsigned int k0, unsigned int k1, int c0)
{
    const int L = g.L;
    for (int r = c0; r < L; r += g.Gc) {
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

// One pass of a warp over the k replicas [base, base + k) of a population of R replicas
// (replica j = base + sub staged in S, the warp's k replicas in Sw): simple sampling (INIT) or
// a load, the theta sweeps, the measurement, the store; the level, magnetisation (and family
// id) of each replica are written.  The group's first lane of an active replica returns its
// level and fills v with its seven exact sums (|M|, M^2, k0, k0^2, k1, k1^2, k0 k1); others
// return -1.
template <bool INIT>
__device__ __forceinline__ int any_pass(const SweepArgs &a, const AnyGeo &g, int L, long long R, long long base,
                                        u64 *Sw, const ClassThr &th, unsigned long long *v)
{
    const int N = L * L, W2 = 2 * L;  // words per replica
    const int lane = threadIdx.x & 31;
    const int sub = lane / g.Gc, c0 = lane % g.Gc;  // replica within the warp, lane within its group
    u64 *S = Sw + sub * W2;
    const int KW = g.k * W2;  // words of the warp's replicas
    const long long j = base + sub;
    const bool active = j < R;
    const unsigned int slot = (unsigned int)j + a.slot_base;  // global replica slot
    // the warp's k replicas are consecutive in HBM; slots past R read as zero
    if (INIT) {
        init_any(S, g, slot, a.k0, a.k1, c0);
    } else if (g.wide) {
        const u64 *src = reinterpret_cast<const u64 *>(a.spins) + (size_t)base * W2;
        for (int w = lane; w < KW; w += 32) Sw[w] = (base + w / W2 < R) ? src[w] : 0ull;
    } else {
        const unsigned int *src = reinterpret_cast<const unsigned int *>(a.spins) + (size_t)base * W2;
        for (int w = lane; w < KW; w += 32) Sw[w] = (base + w / W2 < R) ? src[w] : 0u;
    }
    __syncwarp();
    for (int t = 0; t < a.theta; ++t)
        for (int q = 0; q < 2; ++q) {
            const unsigned int tag = (unsigned int)(2 * (a.t0 + t) + q);
            if (g.wide) half_sweep_rows(S, g, q, slot, tag, a.step, a.k0, a.k1, th, c0);
            else half_sweep_chunks(S, g, q, slot, tag, a.step, a.k0, a.k1, th, c0);
            __syncwarp();
        }
    // measurement: antiparallel bonds (row r: (2p, 2p+1), (2p+1, 2p+2); column: r, r+1)
    int anti = 0, ups = 0;
    for (int r = c0; r < L; r += g.Gc) {
        const int rn = (r == L - 1) ? 0 : r + 1;
        const u64 E = S[2 * r], O = S[2 * r + 1];
        const u64 En = ((E >> 1) | (E << (g.H - 1))) & g.hmask;
        anti += __popcll(E ^ O) + __popcll(O ^ En) + __popcll(E ^ S[2 * rn]) + __popcll(O ^ S[2 * rn + 1]);
        ups += __popcll(E) + __popcll(O);
    }
    for (int o = g.Gc / 2; o > 0; o >>= 1) {  // sum over the replica's lane group
        anti += __shfl_xor_sync(0xffffffffu, anti, o);
        ups += __shfl_xor_sync(0xffffffffu, ups, o);
    }
    if (INIT || a.theta > 0) {
        if (g.wide) {
            u64 *dst = reinterpret_cast<u64 *>(a.spins) + (size_t)base * W2;
            for (int w = lane; w < KW; w += 32)
                if (base + w / W2 < R) dst[w] = Sw[w];
        } else {
            unsigned int *dst = reinterpret_cast<unsigned int *>(a.spins) + (size_t)base * W2;
            for (int w = lane; w < KW; w += 32)
                if (base + w / W2 < R) dst[w] = (unsigned int)Sw[w];
        }
    }
    __syncwarp();  // the stores have read S before the next replicas overwrite it
    if (c0 != 0 || !active) return -1;
    const int level = anti >> 1;
    const int M = 2 * ups - N;
    v[0] = (unsigned long long)(M < 0 ? -M : M);
    v[1] = (unsigned long long)((long long)M * M);
    for (int i = 2; i < 7; ++i) v[i] = 0;
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
    if (INIT) a.fam[j] = (int)slot;
    return level;
}

template <bool INIT>
__global__ void __launch_bounds__(32 * kAnyWarps, PA_ANY_MIN_BLOCKS) k_sweep_any(SweepArgs a, int L)
{
    const AnyGeo g = any_geo(L);
    extern __shared__ u64 sh_dyn[];
    const int N = L * L, W2 = 2 * L;  // words per replica
    u64 *Sw = sh_dyn + (size_t)(threadIdx.x >> 5) * g.k * W2;  // the warp's k replicas
    int *sh_hist = reinterpret_cast<int *>(sh_dyn + (size_t)kAnyWarps * g.k * W2);
    __shared__ unsigned long long sh_sum[7];
    for (int k = threadIdx.x; k <= N; k += blockDim.x) sh_hist[k] = 0;
    if (threadIdx.x < 7) sh_sum[threadIdx.x] = 0;
    __syncthreads();

    const long long R = INIT ? a.R_init : a.st->R_cur;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const ClassThr th = class_thresholds(a.update, a.T4, a.T8);
    if (!INIT && blockIdx.x == 0 && threadIdx.x == 0 && (a.T4 != a.st->T4 || a.T8 != a.st->T8))
        set_error(a.st, PA_ERR_NUMERIC);  // host and device thresholds disagree (never expected)

    for (long long base = warp * g.k; base < R; base += nwarps * g.k) {
        unsigned long long v[7];
        const int level = any_pass<INIT>(a, g, L, R, base, Sw, th, v);
        if (level >= 0) {
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

// Batched form: a persistent sweep over the work items of the batch's runs without a register
// kernel (group kBatchAnyGroup); an item is ipw warp passes (k replicas each) of one run, whose
// buffers, key and thresholds come from its sweep descriptor (BatchDesc, written for the step
// by k_b_items); levels go to the run's histogram, the seven sums once per item.  Dry
// (autotuning) launches do nothing.
__global__ void __launch_bounds__(32 * kAnyWarps, PA_ANY_MIN_BLOCKS) k_b_sweep_any(BatchCtl *ctl,
                                                                                const long long *item_start,
                                                                                int max_kw)
{
    extern __shared__ u64 sh_dyn[];
    if (ctl->dry) return;
    const int lane = threadIdx.x & 31;
    u64 *Sw = sh_dyn + (size_t)(threadIdx.x >> 5) * max_kw;
    const long long end = ctl->end[kBatchAnyGroup];
    const int p0 = ctl->pbeg[kBatchAnyGroup], p1 = ctl->pend[kBatchAnyGroup];
    const BatchDesc *desc = ctl->desc;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(&ctl->next[kBatchAnyGroup], 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= end) break;
        const BatchDesc &d = desc[item_position(item_start, item, p0, p1)];
        const SweepArgs a = d.a;
        const int L = d.L;
        const AnyGeo g = any_geo(L);
        const ClassThr th = class_thresholds(a.update, a.T4, a.T8);
        const long long R = d.R;
        const long long it = item - d.item0;
        const int ipw = d.ipw;
        unsigned long long acc[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < ipw; ++k) {
            const long long base = (it * ipw + k) * g.k;
            if (base >= R) break;  // uniform over the warp
            unsigned long long v[7];
            const int level = any_pass<false>(a, g, L, R, base, Sw, th, v);
            if (level >= 0) {
                atomicAdd(&a.hist[level], 1);
                for (int i = 0; i < 7; ++i) acc[i] += v[i];
            }
        }
        for (int i = 0; i < 7; ++i)
            for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        if (lane == 0) {
            atomicAdd(&a.st->sum_absM, acc[0]);
            atomicAdd(&a.st->sum_M2, acc[1]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c0), acc[2]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c00), acc[3]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c1), acc[4]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c11), acc[5]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.st->c01), acc[6]);
        }
    }
}

// shared memory of a block: the replicas of its warps, then the level histogram
size_t any_smem_bytes(int L)
{
    return (size_t)kAnyWarps * any_geo(L).k * 2 * L * sizeof(u64) + (size_t)(L * L + 1) * sizeof(int);
}

template <bool INIT>
cudaError_t launch_any_t(int L, const SweepArgs &a, int num_sms, cudaStream_t s)
{
    const size_t smem = any_smem_bytes(L);
    static PerDeviceOnce once;  // the limit is set once per device, for the largest need
    cudaError_t e = once([] {
        size_t most = 0;
        for (int l = 4; l <= 128; l += 2) most = any_smem_bytes(l) > most ? any_smem_bytes(l) : most;
        return cudaFuncSetAttribute(k_sweep_any<INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    });
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_any<INIT>, 32 * kAnyWarps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long per_block = (long long)kAnyWarps * any_geo(L).k;  // replicas per block and pass
    long long blocks = (a.R_bound + per_block - 1) / per_block;
    const long long cap = (long long)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_sweep_any<INIT><<<(unsigned int)blocks, 32 * kAnyWarps, smem, s>>>(a, L);
    return cudaGetLastError();
}

}  // namespace

int any_replicas_per_pass(int L) { return any_geo(L).k; }
int any_warp_words(int L) { return any_geo(L).k * 2 * L; }
size_t batch_any_smem(int max_kw) { return (size_t)kAnyWarps * max_kw * sizeof(u64); }

cudaError_t prepare_batch_sweep_any(size_t smem)
{
    return cudaFuncSetAttribute(k_b_sweep_any, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int batch_any_blocks_per_sm(size_t smem)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_b_sweep_any, 32 * kAnyWarps, smem) != cudaSuccess) return 1;
    return b > 0 ? b : 1;
}

cudaError_t launch_batch_sweep_any(BatchCtl *ctl, const long long *item_start, int grid, int max_kw, cudaStream_t s)
{
    k_b_sweep_any<<<grid, 32 * kAnyWarps, batch_any_smem(max_kw), s>>>(ctl, item_start, max_kw);
    return cudaGetLastError();
}

cudaError_t launch_sweep_any(int L, bool init, const SweepArgs &a, int num_sms, cudaStream_t s)
{
    if (L < 4 || L > 128 || (L & 1)) return cudaErrorInvalidValue;
    return init ? launch_any_t<true>(L, a, num_sms, s) : launch_any_t<false>(L, a, num_sms, s);
}

}  // namespace pa
