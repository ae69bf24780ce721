// pa_sweep.cuh -- step 1 (simple-sampling initialisation) and step 3 (theta checkerboard
// Metropolis sweeps) of population annealing (arXiv:2102.06611, Sec. II), each fused with
// the measurement of step 4 (energy level, magnetisation, level histogram, exact sums).
//
// One replica is held entirely in registers by G lanes of a warp (lane g owns RPL rows,
// two half-row words per row), so all theta sweeps run without touching memory: a replica
// is read once and written once per call.  Neighbouring rows owned by other lanes come in
// through warp shuffles.  The update of one colour of one row is bit-sliced over the whole
// half-row word: aligned-neighbour classes come from XORs with the four neighbour words, and
// only the acceptance bits need per-site random numbers.
//
// Metropolis rule (Sec. IV, acceptance min[1, exp(-beta dE)], dE = 4a - 8 for a aligned
// neighbours): a <= 2 flips; a = 3 flips iff x < floor(e^{-4 beta} 2^32); a = 4 flips iff
// x < floor(e^{-8 beta} 2^32), with x a uniform 32-bit integer per site drawn from Philox
// (key = seed): its top 8 bits come from bit planes shared by the 32 sites of a word, its low
// 24 bits from a per-site draw made only when the top bits tie with the threshold (see
// half_sweep for the counters).
#pragma once

#include "pa_common.cuh"
#include "pa_kernels.h"

// Block shape of the sweep kernel, set to the measured best: one block per SM of 512 threads
// (16 warps, at most 128 registers), except L = 128: 384 threads (12 warps, at most 170
// registers; also taken by the other 64-bit-word sizes, 80 and 96, which spill at 128).  Measured at beta = 0.2 / 0.44 / 0.8 against two blocks of 256 per SM (one at
// L = 8 and 128), the previous shape: +3 to +7 % at every size (L = 64 +4.5 %, L = 16 +7 %),
// L = 128 +5.7 % with 384 threads (+1 % with 512); 320, 448 and 640 threads and two blocks of
// 192 or three of 128 were slower.  PA_SWEEP_THREADS / PA_SWEEP_MIN_BLOCKS override the shape
// for every size (build knobs).
#ifdef PA_SWEEP_THREADS
constexpr int sweep_threads(int) { return PA_SWEEP_THREADS; }
#else
constexpr int sweep_threads(int L) { return L >= 80 ? 384 : 512; }
#endif
#ifndef PA_SWEEP_MIN_BLOCKS
#define PA_SWEEP_MIN_BLOCKS 1
#endif
constexpr int sweep_min_blocks(int) { return PA_SWEEP_MIN_BLOCKS; }
#ifndef PA_TM_IMAD
#define PA_TM_IMAD 1   // threshold bits by multiply-add (see Accept)
#endif
#ifndef PA_PREFETCH_MAX_C
#define PA_PREFETCH_MAX_C 3
#endif


namespace pa {

template <typename W, int H>
__device__ __forceinline__ W half_mask()
{
    if constexpr (H == 8 * (int)sizeof(W)) return ~W(0);
    else return (W(1) << H) - W(1);
}

// bit j <- bit j-1 (periodic in H bits)
template <typename W, int H>
__device__ __forceinline__ W rot_up(W x)
{
    return ((x << 1) | (x >> (H - 1))) & half_mask<W, H>();
}

// bit j <- bit j+1 (periodic in H bits)
template <typename W, int H>
__device__ __forceinline__ W rot_down(W x)
{
    return ((x >> 1) | (x << (H - 1))) & half_mask<W, H>();
}

__device__ __forceinline__ int popc(unsigned int x) { return __popc(x); }
__device__ __forceinline__ int popc(unsigned long long x) { return __popcll(x); }

// Philox4x32-10 for calls that differ only in c0.  After round 1 the words 0 and 1 are
// u0 = hi(M1 c2) ^ c1 ^ k0 and u1 = lo(M1 c2), the same for every call, so round 2's
// product M0 * u0 = (v_hi, v_lo) is shared too; u2 = c3 ^ k1, u1k = u1 ^ k0'.
struct PhiloxC0 {
    unsigned int u0, u1, u2;
    unsigned int v_hi, v_lo;
    unsigned int u1k;  // u1 ^ (round-2 key word 0)
};

// Philox4x32-10 with the round keys precomputed (rk[i] = k + i W).
template <bool SPLIT = (PA_MULHI_SPLIT != 0)>
__device__ __forceinline__ uint4 philox_rk_t(uint4 c, const unsigned int *rk0, const unsigned int *rk1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        unsigned int hi0, lo0, hi1, lo1;
        mulhilo<SPLIT>(kPhiloxM0, c.x, hi0, lo0);
        mulhilo<SPLIT>(kPhiloxM1, c.z, hi1, lo1);
        c = make_uint4(hi1 ^ c.y ^ rk0[i], lo1, hi0 ^ c.w ^ rk1[i], lo0);
    }
    return c;
}

// RK: the calls written as plain rounds instead (the compiler then finds the shared part
// itself); faster at some sizes, slower at others (SweepStyle::PLANE_RK, measured).
template <bool SPLIT = (PA_MULHI_SPLIT != 0), bool RK = false>
__device__ __forceinline__ PhiloxC0 philox_c0_setup(unsigned int c1, unsigned int c2, unsigned int c3,
                                                    const unsigned int *rk0, const unsigned int *rk1)
{
    PhiloxC0 p;
    if constexpr (RK) {
        p.u0 = c1;
        p.u1 = c2;
        p.u2 = c3;
        return p;
    }
    unsigned int h1, l1;
    mulhilo<SPLIT>(kPhiloxM1, c2, h1, l1);
    p.u0 = h1 ^ c1 ^ rk0[0];
    p.u1 = l1;
    p.u2 = c3 ^ rk1[0];
    mulhilo<SPLIT>(kPhiloxM0, p.u0, p.v_hi, p.v_lo);
    p.u1k = p.u1 ^ rk0[1];
    return p;
}

template <bool SPLIT = (PA_MULHI_SPLIT != 0), bool RK = false>
__device__ __forceinline__ uint4 philox_c0(unsigned int c0, const PhiloxC0 &p, const unsigned int *rk0,
                                           const unsigned int *rk1)
{
    if constexpr (RK) return philox_rk_t<SPLIT>(make_uint4(c0, p.u0, p.u1, p.u2), rk0, rk1);
    unsigned int hi0, lo0;
    mulhilo<SPLIT>(kPhiloxM0, c0, hi0, lo0);
    // round 1: (u0, u1, hi0 ^ c3 ^ k1, lo0); round 2 with the shared M0 * u0
    const unsigned int z2 = hi0 ^ p.u2, z3 = lo0;
    unsigned int h1, l1;
    mulhilo<SPLIT>(kPhiloxM1, z2, h1, l1);
    uint4 c = make_uint4(h1 ^ p.u1k, l1, p.v_hi ^ z3 ^ rk1[1], p.v_lo);
#pragma unroll
    for (int i = 2; i < 10; ++i) {
        unsigned int h0, l0, h1, l1;
        mulhilo<SPLIT>(kPhiloxM0, c.x, h0, l0);
        mulhilo<SPLIT>(kPhiloxM1, c.z, h1, l1);
        c = make_uint4(h1 ^ c.y ^ rk0[i], l1, h0 ^ c.w ^ rk1[i], l0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_rk(uint4 c, const unsigned int *rk0, const unsigned int *rk1)
{
    return philox_rk_t<>(c, rk0, rk1);
}

// Load / store the RPL rows of one lane as (A, B) pairs: A_r = half (r & 1) of row r (the
// half updated by colour 0), B_r = the other half (updated by colour 1).
template <int L>
__device__ __forceinline__ void load_rows(const typename Geo<L>::W *rep, int r0,
                                          typename Geo<L>::W *A, typename Geo<L>::W *B)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    W w[2 * Gm::RPL];
    const W *src = rep + 2 * r0;
    constexpr int LANE_BYTES = 2 * Gm::RPL * (int)sizeof(W);
    if constexpr (LANE_BYTES % 16 == 0) {
#pragma unroll
        for (int v = 0; v < LANE_BYTES / 16; ++v) {
            uint4 x = reinterpret_cast<const uint4 *>(src)[v];
            reinterpret_cast<uint4 *>(w)[v] = x;
        }
    } else {
#pragma unroll
        for (int v = 0; v < LANE_BYTES / 8; ++v) {
            uint2 x = reinterpret_cast<const uint2 *>(src)[v];
            reinterpret_cast<uint2 *>(w)[v] = x;
        }
    }
#pragma unroll
    for (int i = 0; i < Gm::RPL; ++i) {
        const bool odd = ((r0 + i) & 1) != 0;
        A[i] = odd ? w[2 * i + 1] : w[2 * i];
        B[i] = odd ? w[2 * i] : w[2 * i + 1];
    }
}

template <int L>
__device__ __forceinline__ void store_rows(typename Geo<L>::W *rep, int r0,
                                           const typename Geo<L>::W *A, const typename Geo<L>::W *B)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    W w[2 * Gm::RPL];
#pragma unroll
    for (int i = 0; i < Gm::RPL; ++i) {
        const bool odd = ((r0 + i) & 1) != 0;
        w[2 * i] = odd ? B[i] : A[i];
        w[2 * i + 1] = odd ? A[i] : B[i];
    }
    W *dst = rep + 2 * r0;
    constexpr int LANE_BYTES = 2 * Gm::RPL * (int)sizeof(W);
    if constexpr (LANE_BYTES % 16 == 0) {
#pragma unroll
        for (int v = 0; v < LANE_BYTES / 16; ++v)
            reinterpret_cast<uint4 *>(dst)[v] = reinterpret_cast<const uint4 *>(w)[v];
    } else {
#pragma unroll
        for (int v = 0; v < LANE_BYTES / 8; ++v)
            reinterpret_cast<uint2 *>(dst)[v] = reinterpret_cast<const uint2 *>(w)[v];
    }
}

// Step 1: the rows of one lane from the INIT stream.  Site n = r L + c is bit n mod 32 of
// 32-bit word n / 32; word w is lane w mod 4 of Philox(ctr = (w / 4, j, INIT << 28, 0)).
template <int L>
__device__ __forceinline__ void init_rows(unsigned int slot, int r0, unsigned int k0, unsigned int k1,
                                          typename Geo<L>::W *A, typename Geo<L>::W *B)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
#pragma unroll 1
    for (int i = 0; i < Gm::RPL; ++i) {
        const int r = r0 + i;
        W E = 0, O = 0;
        unsigned int cached_call = 0xffffffffu;
        uint4 x = make_uint4(0, 0, 0, 0);
#pragma unroll 1
        for (int c = 0; c < L; ++c) {
            const unsigned int n = (unsigned int)(r * L + c);
            const unsigned int w = n >> 5;
            if ((w >> 2) != cached_call) {
                cached_call = w >> 2;
                x = philox(make_uint4(cached_call, slot, kStreamInit << 28, 0u), k0, k1);
            }
            const unsigned int word = (w & 3) == 0 ? x.x : (w & 3) == 1 ? x.y : (w & 3) == 2 ? x.z : x.w;
            const W bit = (W)((word >> (n & 31)) & 1u);
            if (c & 1) O |= bit << (c >> 1);
            else E |= bit << (c >> 1);
        }
        const bool odd = (r & 1) != 0;
        A[i] = odd ? O : E;
        B[i] = odd ? E : O;
    }
}

// ------------------------------------------------------------------------------------
// The Metropolis test on one 32-site word.
//
// Neighbour classes: a site with a aligned neighbours flips always for a <= 2, with the
// class-3 threshold T4 for a = 3 and with T8 for a = 4.  Two equivalent Boolean
// formulations are used, chosen per lattice size because nvcc turns them into code of
// different speed depending on the word layout (measured): XNOR masks of the four
// neighbours with an explicit always-accept mask for T = 2^32, or pair masks (any / exactly
// one antiparallel per pair of neighbours) with T = 2^32 folded into the threshold.
// ------------------------------------------------------------------------------------
template <int L>
struct SweepStyle {
    // neighbour classes by the pair-mask form at every size: with one block of 512 threads per
    // SM and plain-round plane calls it measured +8 % (L = 24), +7 % (48), +3 % (64), +2 % (32)
    // against the XNOR form there and equal elsewhere (the XNOR form had been the faster at
    // L = 24 - 64 with two blocks of 256)
    static constexpr bool XNOR = false;
    // ties resolved through the warp's queue (below) when a lane holds 3 or more words;
    // with 1 or 2 words the lane's own loop is cheaper (measured)
    static constexpr int WORDS = Geo<L>::PACK ? Geo<L>::C : Geo<L>::RPL;
    static constexpr bool TIE_QUEUE = WORDS >= 3;
    static constexpr int TQ_LEN = TIE_QUEUE ? 32 * WORDS : 1;  // queue entries per warp
    // Philox products of the bit planes as separate low/high multiplies (faster from L = 32
    // up, measured) or one widening multiply
    static constexpr bool SPLIT_MUL = (PA_MULHI_SPLIT != 0) && L >= 32;
    // bit-plane calls as plain rounds (philox_c0's RK): +2 % at L = 32, +1.4 % at L = 64, within
    // 1 % at L = 8, 16, 24, 48 and -2.6 % at L = 128 (measured)
    static constexpr bool PLANE_RK = (L == 32 || L == 64);
};

// the plane-call form of an update: the heatbath kernel at L = 64 is 1.7 % faster with the
// shared-round form (at L = 32 the two are within 0.4 %; measured)
template <int L, bool HB>
__host__ __device__ constexpr bool plane_rk()
{
    return SweepStyle<L>::PLANE_RK && !(HB && L == 64);
}


// Per-launch constants.  T = floor(e^{-4 beta} 2^32) (class a = 3) or floor(e^{-8 beta} 2^32)
// (a = 4), T in [0, 2^32], split as T = top 2^24 + low: m[k] = all ones iff bit 7 - k of top
// is set (k = 0 most significant).  T = 2^32 (beta = 0) is either the always-accept mask alw
// (XNOR style, top = low = 0) or top = 255, low = 2^24 (x < 2^32 holds, and so does the
// split test: x_top < 255, or x_top = 255 and x_low < 2^24).
//
// The threshold bit of a site, tm = m8[k] where all4 is set, else m4[k], is also
// all4 * sel[k] + m4[k] (mod 2^32) with sel[k] = 0 where m4[k] = m8[k], +1 where only m8[k]
// is set and -1 where only m4[k] is (then tm = -all4 - 1 = ~all4): one integer multiply-add,
// which issues on the FMA pipe and leaves the logic pipe (the busiest unit of the sweep) to
// the borrow chain (64-bit words: one per 32-bit half).
template <typename W>
struct Accept {
    W m4[8], m8[8];
    W alw4, alw8;
    unsigned int low4, low8;
    unsigned int sel[8];
};

template <typename W>
__device__ __forceinline__ W threshold_bits(W cls, const Accept<W> &ac, int k)
{
#if PA_TM_IMAD
    if constexpr (sizeof(W) == 4) {
        return cls * ac.sel[k] + ac.m4[k];
    } else {  // two 32-bit halves
        const unsigned int m = (unsigned int)ac.m4[k];
        const unsigned int lo = (unsigned int)cls * ac.sel[k] + m, hi = (unsigned int)(cls >> 32) * ac.sel[k] + m;
        return ((W)hi << 32) | (W)lo;
    }
#else
    return (cls & ac.m8[k]) | (~cls & ac.m4[k]);
#endif
}

template <int L>
__device__ __forceinline__ Accept<typename Geo<L>::W> make_accept(unsigned long long T4, unsigned long long T8)
{
    using W = typename Geo<L>::W;
    Accept<W> c;
    const bool all4 = T4 >= (1ull << 32), all8 = T8 >= (1ull << 32);
    unsigned int top4, top8;
    if constexpr (SweepStyle<L>::XNOR) {
        const unsigned int t4 = all4 ? 0u : (unsigned int)T4, t8 = all8 ? 0u : (unsigned int)T8;
        top4 = t4 >> 24;
        top8 = t8 >> 24;
        c.low4 = t4 & 0xFFFFFFu;
        c.low8 = t8 & 0xFFFFFFu;
        c.alw4 = all4 ? ~W(0) : W(0);
        c.alw8 = all8 ? ~W(0) : W(0);
    } else {
        top4 = all4 ? 255u : (unsigned int)(T4 >> 24);
        top8 = all8 ? 255u : (unsigned int)(T8 >> 24);
        c.low4 = all4 ? (1u << 24) : (unsigned int)(T4 & 0xFFFFFFu);
        c.low8 = all8 ? (1u << 24) : (unsigned int)(T8 & 0xFFFFFFu);
        c.alw4 = W(0);
        c.alw8 = W(0);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const unsigned int b4 = (top4 >> (7 - k)) & 1u, b8 = (top8 >> (7 - k)) & 1u;
        c.m4[k] = b4 ? ~W(0) : W(0);
        c.m8[k] = b8 ? ~W(0) : W(0);
        c.sel[k] = (b4 == b8) ? 0u : (b8 ? 1u : 0xFFFFFFFFu);
    }
    return c;
}

// Classes of the sites of word s with neighbour words up, dn, ha, hb (bits outside `valid`
// are cleared): all4 = four aligned neighbours, eq3 = exactly three, ge3 = all4 | eq3.
template <bool XNOR, typename W>
__device__ __forceinline__ void classify(W s, W up, W dn, W ha, W hb, W valid, W &all4, W &eq3, W &ge3)
{
    if constexpr (XNOR) {
        const W x1 = ~(s ^ up), x2 = ~(s ^ dn), x3 = ~(s ^ ha), x4 = ~(s ^ hb);
        all4 = x1 & x2 & x3 & x4 & valid;
        ge3 = ((x1 & x2 & (x3 | x4)) | (x3 & x4 & (x1 | x2))) & valid;
        eq3 = ge3 & ~all4;
    } else {
        // with y_n = s ^ n (antiparallel): z = y_1 | y_2 (any of the pair) and
        // x = y_1 ^ y_2 = n_1 ^ n_2 (exactly one of the pair)
        const W z12 = (s ^ up) | (s ^ dn), x12 = up ^ dn;
        const W z34 = (s ^ ha) | (s ^ hb), x34 = ha ^ hb;
        all4 = ~(z12 | z34) & valid;
        eq3 = ((x12 & ~z34) | (x34 & ~z12)) & valid;
        ge3 = all4 | eq3;
    }
}

// x_top < T_top for every site of classes a = 3, 4 from the 8 bit planes, as a borrow chain
// from the least significant plane (borrow = majority of ~x_k, t_k and the incoming borrow):
// lt = decided accepts, eq = ties x_top = T_top (decided by the low 24 bits).
template <bool XNOR, typename W>
__device__ __forceinline__ void compare_planes(const W *plane, W all4, W eq3, W ge3, const Accept<W> &ac, W &lt,
                                               W &eq)
{
    W dec = 0;
    if constexpr (XNOR) dec = (eq3 & ac.alw4) | (all4 & ac.alw8);
    W l = 0, e = XNOR ? (ge3 & ~dec) : ge3;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const W tm = threshold_bits(all4, ac, k);  // threshold bit of each site
        const W np = ~plane[k];
        l = (np & tm) | (np & l) | (tm & l);
        e &= ~(plane[k] ^ tm);
    }
    lt = XNOR ? (l | dec) : l;
    eq = e;
}

// Heatbath (Sec. IV): every site draws; with A = 4 - a antiparallel neighbours the classes
// are c04 (A = 0 or 4: threshold T_4, x for A = 0 / ~x for A = 4), c13 (A = 1 or 3:
// threshold T_3), clow (A >= 3, the sites that compare ~x) and c2 (A = 2: flip iff the top
// bit of x is 0, x < 2^31).  With pair masks z = y_1 | y_2, x = y_1 ^ y_2, d = y_1 & y_2 of
// y_n = s ^ n: A = 0 is ~z12 & ~z34, A = 4 is d12 & d34, A >= 3 is (d12 & z34) | (x12 & d34),
// A = 2 is (d12 & ~z34) | (x12 & x34) | (~z12 & d34).
template <typename W>
__device__ __forceinline__ void classify_hb(W s, W up, W dn, W ha, W hb, W valid, W &c04, W &clow, W &c2)
{
    const W y1 = s ^ up, y2 = s ^ dn, y3 = s ^ ha, y4 = s ^ hb;
    const W z12 = y1 | y2, x12 = up ^ dn, d12 = y1 & y2;
    const W z34 = y3 | y4, x34 = ha ^ hb, d34 = y3 & y4;
    c04 = ((~z12 & ~z34) | (d12 & d34)) & valid;
    clow = ((d12 & z34) | (x12 & d34)) & valid;
    c2 = ((d12 & ~z34) | (x12 & x34) | (~z12 & d34)) & valid;
}

// The heatbath decision from the 8 planes: x' = x (A <= 1) or ~x (A >= 3) against T (T_4 for
// c04, T_3 otherwise) by the borrow chain; a site flips iff x' < T for A <= 1 and iff
// x' >= T (~x >= T, i.e. x < 2^32 - T) for A >= 3; A = 2 flips iff plane 0 (bit 31 of x) is 0.
// flip = the decided flips (for ties x'_top = T_top it holds the decision for x'_low >= T_low,
// which the tie resolution toggles where x'_low < T_low), eq = the ties.
template <typename W>
__device__ __forceinline__ void compare_planes_hb(const W *plane, W c04, W clow, W c2, W valid, const Accept<W> &ac,
                                                  W &flip, W &eq)
{
    W l = 0, e = ~c2 & valid;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const W tm = threshold_bits(c04, ac, k);
        const W pp = plane[k] ^ clow;
        const W np = ~pp;
        l = (np & tm) | (np & l) | (tm & l);
        e &= ~(pp ^ tm);
    }
    flip = ((c2 & ~plane[0]) | (~c2 & (l ^ clow))) & valid;
    eq = e;
}

// ------------------------------------------------------------------------------------
// Ties x_top = T_top are rare (2^-8 per site) but land on few lanes of a warp, so a loop in
// which every lane resolves its own ties runs as many Philox passes as the busiest lane has
// ties.  Instead the warp resolves them together: every (lane, word) with ties becomes one
// entry of a per-warp queue in shared memory, lane t draws the low bits of the sites of entry
// t (t + 32, ... if there are more), and the owners read the accept bits back.  One pass
// usually serves the whole warp.
// ------------------------------------------------------------------------------------
template <typename W>
struct TieQueue {
    W *eq;              // tie mask of the entry's word (overwritten with the accept mask)
    W *a4;              // sites compared with the second threshold (class 4 / heatbath c04)
    W *inv;             // heatbath: sites that compare the complemented low bits (else unused)
    unsigned int *code; // owner lane << 4 | word index
};

struct TieSite {
    unsigned int slot;  // replica slot
    int r, j;           // row and position within the colour's half-row
};

// For entry t the accept mask has bit b set iff x_low < thr (low8 where a4 is set, else
// low4), with x_low the low 24 bits of the site's refinement draw, complemented where inv is
// set (heatbath, HB).  The owners XOR it into `flip` (zero at the ties for Metropolis).
template <int NW, bool HB, typename W, typename SiteOf>
__device__ __forceinline__ void resolve_ties(const W *eq, const W *a4, const W *inv, W *flip, int lane,
                                             const TieQueue<W> &q, SiteOf site_of, unsigned int tag,
                                             unsigned int step, const unsigned int *rk0, const unsigned int *rk1,
                                             unsigned int low4, unsigned int low8)
{
    static_assert(NW <= 15, "word index is 4 bits of the entry code");
    const unsigned int below = (1u << lane) - 1u;
    int pos[NW];
    int total = 0;
    __syncwarp();  // the previous call's read-back is complete
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const unsigned int b = __ballot_sync(0xffffffffu, eq[i] != W(0));
        pos[i] = total + __popc(b & below);
        if (eq[i] != W(0)) {
            q.eq[pos[i]] = eq[i];
            q.a4[pos[i]] = a4[i];
            if constexpr (HB) q.inv[pos[i]] = inv[i];
            q.code[pos[i]] = ((unsigned int)lane << 4) | (unsigned int)i;
        }
        total += __popc(b);
    }
    if (total == 0) return;
    __syncwarp();
    for (int t = lane; t < total; t += 32) {
        W w = q.eq[t];
        const W a = q.a4[t];
        W v = 0;
        if constexpr (HB) v = q.inv[t];
        const unsigned int code = q.code[t];
        W acc = 0;
        while (w) {
            const int b = (sizeof(W) == 8) ? __ffsll((long long)w) - 1 : __ffs((int)w) - 1;
            const TieSite s = site_of((int)(code >> 4), (int)(code & 15u), b);
            const uint4 x = philox_rk(make_uint4((unsigned int)(64 * s.r + s.j), s.slot, (kStreamRefine << 28) | tag,
                                                 step), rk0, rk1);
            const unsigned int thr = ((a >> b) & W(1)) ? low8 : low4;
            unsigned int xl = x.x & 0xFFFFFFu;
            if (HB && ((v >> b) & W(1))) xl ^= 0xFFFFFFu;
            if (xl < thr) acc |= W(1) << b;
            w &= w - W(1);
        }
        q.eq[t] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NW; ++i)
        if (eq[i] != W(0)) flip[i] ^= q.eq[pos[i]];
}

// One colour (compile-time Q) of one sweep over the rows a lane holds (sizes L >= 48).
//
// Acceptance x < T is decided over the 32 sites of a word at once: the top 8 bits of every
// site's uniform x are 8 bit planes (bit j of plane k is bit 31 - k of site j's x); a site
// stays undecided only if its top bits equal the threshold's, which happens with
// probability 2^-8, and only then is its low 24-bit part drawn.  Plane k of row r is word
// k mod 4 of Philox(ctr = (2 (nh r + h) + k / 4, slot, SWEEP << 28 | tag, i)) for the 32-site
// chunk h of the half-row (nh = chunks per half-row); the low part of site j is the low 24
// bits of word 0 of Philox(ctr = (64 r + j, slot, REFINE << 28 | tag, i)), tag = 2t + Q.
template <int L, int Q, bool HB>
__device__ __forceinline__ void half_sweep(typename Geo<L>::W *A, typename Geo<L>::W *B, int r0,
                                           int lane, unsigned int slot, unsigned int slot0, unsigned int tag,
                                           unsigned int step, const unsigned int *rk0,
                                           const unsigned int *rk1, const Accept<typename Geo<L>::W> &ac,
                                           const TieQueue<typename Geo<L>::W> &tq)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    constexpr int RPL = Gm::RPL, G = Gm::G, H = Gm::H;
    constexpr int NH = Gm::WIDE ? 2 : 1;  // 32-site chunks per half-row
    constexpr bool XNOR = SweepStyle<L>::XNOR;
    W *T = (Q == 0) ? A : B;          // words updated by this colour
    const W *O = (Q == 0) ? B : A;    // the other half of each row (read only here)

    // rows r0 - 1 and r0 + RPL come from the neighbouring lanes of the group
    const int gbase = lane & ~(G - 1);
    const int q = lane & (G - 1);
    const W from_up = __shfl_sync(0xffffffffu, O[RPL - 1], gbase | ((q - 1) & (G - 1)));
    const W from_down = __shfl_sync(0xffffffffu, O[0], gbase | ((q + 1) & (G - 1)));

    // the plane stream's calls differ only in c0 (rounds 1 and 2 partly shared)
    constexpr bool SM = SweepStyle<L>::SPLIT_MUL, RK = plane_rk<L, HB>();
    const PhiloxC0 pc = philox_c0_setup<SM, RK>(slot, (kStreamSweep << 28) | tag, step, rk0, rk1);

    // Metropolis: lt = decided accepts, g3 = sites with a >= 3; heatbath: lt = flip, g3 = clow
    W lt[RPL], eq[RPL], a4[RPL], g3[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const int r = r0 + i;
        const W up = (i == 0) ? from_up : O[i - 1];
        const W dn = (i == RPL - 1) ? from_down : O[i + 1];
        // the updated half is the even-column half iff (r + Q) is even
        const bool even_half = ((r + Q) & 1) == 0;
        const W hb = even_half ? rot_up<W, H>(O[i]) : rot_down<W, H>(O[i]);
        W all4, eq3, ge3, c2;
        if constexpr (HB) classify_hb(T[i], up, dn, O[i], hb, half_mask<W, H>(), all4, ge3, c2);
        else classify<XNOR>(T[i], up, dn, O[i], hb, half_mask<W, H>(), all4, eq3, ge3);

        // bit planes of the top 8 bits of every site's uniform
        W plane[8];
        if constexpr (NH == 1) {
            const uint4 p0 = philox_c0<SM, RK>((unsigned int)(2 * r), pc, rk0, rk1);
            const uint4 p1 = philox_c0<SM, RK>((unsigned int)(2 * r + 1), pc, rk0, rk1);
            plane[0] = p0.x; plane[1] = p0.y; plane[2] = p0.z; plane[3] = p0.w;
            plane[4] = p1.x; plane[5] = p1.y; plane[6] = p1.z; plane[7] = p1.w;
        } else {
            const uint4 a0 = philox_c0<SM, RK>((unsigned int)(4 * r), pc, rk0, rk1);
            const uint4 a1 = philox_c0<SM, RK>((unsigned int)(4 * r + 1), pc, rk0, rk1);
            const uint4 b0 = philox_c0<SM, RK>((unsigned int)(4 * r + 2), pc, rk0, rk1);
            const uint4 b1 = philox_c0<SM, RK>((unsigned int)(4 * r + 3), pc, rk0, rk1);
            const unsigned int lo[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const unsigned int hi[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) plane[k] = (W)lo[k] | ((W)hi[k] << 32);
        }
        if constexpr (HB) compare_planes_hb(plane, all4, ge3, c2, half_mask<W, H>(), ac, lt[i], eq[i]);
        else compare_planes<XNOR>(plane, all4, eq3, ge3, ac, lt[i], eq[i]);
        a4[i] = all4;
        g3[i] = ge3;
    }

    // rare: the low 24 bits decide the sites whose top 8 bits equal the threshold's
    static_assert(SweepStyle<L>::TIE_QUEUE, "row-wise sizes hold 3 or more words per lane");
    (void)slot;
    resolve_ties<RPL, HB>(eq, a4, g3, lt, lane, tq,
                          [&](int src, int i, int b) {
                              return TieSite{slot0 + (unsigned int)(src / G), (src & (G - 1)) * RPL + i, b};
                          },
                          tag, step, rk0, rk1, ac.low4, ac.low8);
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        if constexpr (HB) T[i] ^= lt[i];
        else T[i] ^= (~g3[i] | lt[i]) & half_mask<W, H>();
    }
}

// ------------------------------------------------------------------------------------
// Packed sizes (L < 48): the P rows of one chunk are one register word, field i (bits
// i H' .. i H' + H - 1) = row (first row of the chunk + i).  PA[c] packs the colour-0 words
// A_r of chunk c, PB[c] the colour-1 words B_r.  The first row of every chunk is even.
// ------------------------------------------------------------------------------------
template <int L>
struct PackMasks {
    using Gm = Geo<L>;
    static constexpr unsigned int field(int i, unsigned int bits) { return bits << (i * Gm::HP); }
    static constexpr unsigned int rep(unsigned int bits, int parity)  // parity -1: every field
    {
        unsigned int m = 0;
        for (int i = 0; i < Gm::P; ++i)
            if (parity < 0 || (i & 1) == parity) m |= field(i, bits);
        return m;
    }
    static constexpr unsigned int VALID = rep((1u << Gm::H) - 1u, -1);
    static constexpr unsigned int LSBF = rep(1u, -1);
    static constexpr unsigned int MSBF = rep(1u << (Gm::H - 1), -1);
    static constexpr unsigned int EVENF = rep(Gm::HP >= 32 ? 0xffffffffu : (1u << Gm::HP) - 1u, 0);
};

template <int L>
__device__ __forceinline__ void pack_rows(const unsigned int *A, const unsigned int *B, unsigned int *PA,
                                          unsigned int *PB)
{
    using Gm = Geo<L>;
#pragma unroll
    for (int c = 0; c < Gm::C; ++c) {
        unsigned int a = 0, b = 0;
#pragma unroll
        for (int i = 0; i < Gm::P; ++i) {
            a |= A[c * Gm::P + i] << (i * Gm::HP);
            b |= B[c * Gm::P + i] << (i * Gm::HP);
        }
        PA[c] = a;
        PB[c] = b;
    }
}

template <int L>
__device__ __forceinline__ void unpack_rows(const unsigned int *PA, const unsigned int *PB, unsigned int *A,
                                            unsigned int *B)
{
    using Gm = Geo<L>;
    constexpr unsigned int m = (1u << Gm::H) - 1u;
#pragma unroll
    for (int c = 0; c < Gm::C; ++c)
#pragma unroll
        for (int i = 0; i < Gm::P; ++i) {
            A[c * Gm::P + i] = (PA[c] >> (i * Gm::HP)) & m;
            B[c * Gm::P + i] = (PB[c] >> (i * Gm::HP)) & m;
        }
}

// The 8 bit planes of the lane's C chunks for one colour and sweep (chunk index = first row
// of the chunk / P): words of Philox(ctr = (2 chunk + k / 4, slot, SWEEP << 28 | tag, i)).
template <int L>
__device__ __forceinline__ void packed_planes(int r0, unsigned int slot, unsigned int tag, unsigned int step,
                                              const unsigned int *rk0, const unsigned int *rk1,
                                              unsigned int (*plane)[8])
{
    using Gm = Geo<L>;
    constexpr bool SM = SweepStyle<L>::SPLIT_MUL, RK = SweepStyle<L>::PLANE_RK;
    const PhiloxC0 pc = philox_c0_setup<SM, RK>(slot, (kStreamSweep << 28) | tag, step, rk0, rk1);
    const unsigned int chunk0 = (unsigned int)(r0 / Gm::P);
#pragma unroll
    for (int c = 0; c < Gm::C; ++c) {
        const unsigned int ch = chunk0 + (unsigned int)c;
        const uint4 p0 = philox_c0<SM, RK>(2 * ch, pc, rk0, rk1);
        const uint4 p1 = philox_c0<SM, RK>(2 * ch + 1, pc, rk0, rk1);
        plane[c][0] = p0.x; plane[c][1] = p0.y; plane[c][2] = p0.z; plane[c][3] = p0.w;
        plane[c][4] = p1.x; plane[c][5] = p1.y; plane[c][6] = p1.z; plane[c][7] = p1.w;
    }
}

// One colour (compile-time Q) of one sweep over the packed chunks of a lane, given that
// colour's bit planes.  The same Metropolis test as half_sweep on 32 sites of P rows per
// word: the vertical neighbours are the other colour's chunk word shifted by one field (the
// field across a chunk boundary comes from the neighbouring chunk, lane or, at G = 1, the
// periodic wrap), the horizontal ones the other colour's word as it is and rotated by one
// site within every field, up in the fields whose row updates its even-column half and down
// in the others.
//
// With PRE the planes come in `plane` (drawn by packed_planes); otherwise they are drawn
// here, chunk by chunk.
template <int L, int Q, bool PRE, bool HB>
__device__ __forceinline__ void packed_update(unsigned int *PA, unsigned int *PB, const unsigned int (*plane)[8],
                                              int r0, int lane, unsigned int slot, unsigned int slot0,
                                              unsigned int tag, unsigned int step, const unsigned int *rk0,
                                              const unsigned int *rk1, const Accept<unsigned int> &ac,
                                              const TieQueue<unsigned int> &tq)
{
    using Gm = Geo<L>;
    using Mk = PackMasks<L>;
    constexpr int C = Gm::C, G = Gm::G, H = Gm::H, HP = Gm::HP, P = Gm::P, CB = Gm::CB;
    constexpr bool XNOR = SweepStyle<L>::XNOR;
    constexpr unsigned int LSBF = Mk::LSBF, MSBF = Mk::MSBF;
    // fields whose row updates its even-column half: rows with (r + Q) even
    constexpr unsigned int SEL_UP = (Q == 0) ? Mk::EVENF : ~Mk::EVENF;
    unsigned int *T = (Q == 0) ? PA : PB;
    const unsigned int *O = (Q == 0) ? PB : PA;

    unsigned int from_up, from_down;
    if constexpr (G > 1) {
        const int gbase = lane & ~(G - 1);
        const int q = lane & (G - 1);
        from_up = __shfl_sync(0xffffffffu, O[C - 1], gbase | ((q - 1) & (G - 1)));
        from_down = __shfl_sync(0xffffffffu, O[0], gbase | ((q + 1) & (G - 1)));
    } else {
        from_up = O[C - 1];
        from_down = O[0];
    }

    PhiloxC0 pc;
    if constexpr (!PRE)
        pc = philox_c0_setup<SweepStyle<L>::SPLIT_MUL, plane_rk<L, HB>()>(slot, (kStreamSweep << 28) | tag,
                                                                                 step, rk0, rk1);

    unsigned int lt[C], eq[C], a4[C], g3[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const unsigned int o = O[c];
        const unsigned int prev = (c == 0) ? from_up : O[c - 1];
        const unsigned int next = (c == C - 1) ? from_down : O[c + 1];
        unsigned int up, dn;
        if constexpr (CB == 32) {
            up = __funnelshift_l(prev, o, HP);   // field i <- field i - 1, field 0 <- prev's last
            dn = __funnelshift_r(o, next, HP);   // field i <- field i + 1, last <- next's field 0
        } else {  // one chunk word holds the whole replica (L = 4): rotate by one field
            constexpr unsigned int all = (1u << CB) - 1u;
            up = ((o << HP) | (o >> (CB - HP))) & all;
            dn = ((o >> HP) | (o << (CB - HP))) & all;
        }
        const unsigned int ru = ((o << 1) & ~LSBF) | ((o >> (H - 1)) & LSBF);  // site j <- j - 1
        const unsigned int rd = ((o >> 1) & ~MSBF) | ((o << (H - 1)) & MSBF);  // site j <- j + 1
        const unsigned int hb = (ru & SEL_UP) | (rd & ~SEL_UP);
        // Metropolis: lt = decided accepts, g3 = sites with a >= 3; heatbath: lt = flip,
        // all4 = c04, g3 = clow
        unsigned int all4, eq3, ge3, c2;
        if constexpr (HB) classify_hb(T[c], up, dn, o, hb, Mk::VALID, all4, ge3, c2);
        else classify<XNOR>(T[c], up, dn, o, hb, Mk::VALID, all4, eq3, ge3);
        unsigned int pl[8];
        if constexpr (PRE) {
#pragma unroll
            for (int k = 0; k < 8; ++k) pl[k] = plane[c][k];
        } else {
            const unsigned int ch = (unsigned int)(r0 / P + c);
            const uint4 p0 = philox_c0<SweepStyle<L>::SPLIT_MUL, plane_rk<L, HB>()>(2 * ch, pc, rk0, rk1);
            const uint4 p1 = philox_c0<SweepStyle<L>::SPLIT_MUL, plane_rk<L, HB>()>(2 * ch + 1, pc, rk0, rk1);
            pl[0] = p0.x; pl[1] = p0.y; pl[2] = p0.z; pl[3] = p0.w;
            pl[4] = p1.x; pl[5] = p1.y; pl[6] = p1.z; pl[7] = p1.w;
        }
        if constexpr (HB) compare_planes_hb(pl, all4, ge3, c2, Mk::VALID, ac, lt[c], eq[c]);
        else compare_planes<XNOR>(pl, all4, eq3, ge3, ac, lt[c], eq[c]);
        a4[c] = all4;
        g3[c] = ge3;
    }

    if constexpr (SweepStyle<L>::TIE_QUEUE) {
        resolve_ties<C, HB>(eq, a4, g3, lt, lane, tq,
                                [&](int src, int c, int b) {
                                return TieSite{slot0 + (unsigned int)(src / G),
                                               (src & (G - 1)) * Gm::RPL + c * P + b / HP, b % HP};
                            },
                            tag, step, rk0, rk1, ac.low4, ac.low8);
    } else {
        // the lane resolves its own ties, one per iteration over all its words
        unsigned int pending = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) pending |= eq[c];
        while (pending) {
            int csel = 0;
            unsigned int w = 0, a4s = 0, invs = 0;
#pragma unroll
            for (int c = C - 1; c >= 0; --c)
                if (eq[c]) {
                    csel = c;
                    w = eq[c];
                    a4s = a4[c];
                    if constexpr (HB) invs = g3[c];
                }
            const int b = __ffs((int)w) - 1;
            const int r = r0 + csel * P + b / HP, j = b % HP;
            const uint4 xr = philox_rk(make_uint4((unsigned int)(64 * r + j), slot, (kStreamRefine << 28) | tag, step),
                                       rk0, rk1);
            const unsigned int thr = ((a4s >> b) & 1u) ? ac.low8 : ac.low4;
            const unsigned int bit = 1u << b;
            unsigned int xl = xr.x & 0xFFFFFFu;
            if (HB && ((invs >> b) & 1u)) xl ^= 0xFFFFFFu;
            const unsigned int acc = (xl < thr) ? bit : 0u;
            pending = 0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (c == csel) {
                    eq[c] &= ~bit;
                    lt[c] ^= acc;
                }
                pending |= eq[c];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if constexpr (HB) T[c] ^= lt[c];
        else T[c] ^= (~g3[c] | lt[c]) & Mk::VALID;
    }
}

// theta sweeps (numbered t0 .. t0 + theta - 1 within the temperature step) of the rows a
// lane holds: on packed chunks for L < 48 and row by row otherwise.  With at most two chunks
// per lane both colours' planes are drawn before either update (they do not depend on the
// spins), which gives the scheduler independent work.
//
// slot = the lane's replica slot, slot0 = the slot of the warp's first replica; tq = the
// warp's tie queue.
template <int L, bool HB>
__device__ __forceinline__ void sweep_rows(typename Geo<L>::W *A, typename Geo<L>::W *B, int r0, int lane,
                                           unsigned int slot, unsigned int slot0, int t0, int theta,
                                           unsigned int step, const unsigned int *rk0, const unsigned int *rk1,
                                           const Accept<typename Geo<L>::W> &ac,
                                           const TieQueue<typename Geo<L>::W> &tq)
{
    using Gm = Geo<L>;
    if constexpr (Gm::PACK) {
        constexpr int C = Gm::C;
        if (theta <= 0) return;
        unsigned int PA[C], PB[C];
        pack_rows<L>(A, B, PA, PB);
#pragma unroll 1
        for (int t = 0; t < theta; ++t) {
            const unsigned int tag0 = (unsigned int)(2 * (t0 + t));
            if constexpr (C <= PA_PREFETCH_MAX_C) {
                unsigned int pl0[C][8], pl1[C][8];
                packed_planes<L>(r0, slot, tag0, step, rk0, rk1, pl0);
                packed_planes<L>(r0, slot, tag0 | 1u, step, rk0, rk1, pl1);
                packed_update<L, 0, true, HB>(PA, PB, pl0, r0, lane, slot, slot0, tag0, step, rk0, rk1, ac, tq);
                packed_update<L, 1, true, HB>(PA, PB, pl1, r0, lane, slot, slot0, tag0 | 1u, step, rk0, rk1, ac, tq);
            } else {
                packed_update<L, 0, false, HB>(PA, PB, nullptr, r0, lane, slot, slot0, tag0, step, rk0, rk1, ac, tq);
                packed_update<L, 1, false, HB>(PA, PB, nullptr, r0, lane, slot, slot0, tag0 | 1u, step, rk0, rk1, ac, tq);
            }
        }
        unpack_rows<L>(PA, PB, A, B);
    } else {
#pragma unroll 1
        for (int t = 0; t < theta; ++t) {
            const unsigned int tag0 = (unsigned int)(2 * (t0 + t));
            half_sweep<L, 0, HB>(A, B, r0, lane, slot, slot0, tag0, step, rk0, rk1, ac, tq);
            half_sweep<L, 1, HB>(A, B, r0, lane, slot, slot0, tag0 | 1u, step, rk0, rk1, ac, tq);
        }
    }
}

// Energy level n_anti / 2 and number of up spins of the rows a lane holds (summed over the
// group by the caller).  Antiparallel bonds: horizontal within a row (even-odd and
// odd-next-even neighbours) and vertical to the next row (A_r ^ B_{r+1}, B_r ^ A_{r+1}).
template <int L>
__device__ __forceinline__ void measure_rows(const typename Geo<L>::W *A, const typename Geo<L>::W *B,
                                             int r0, int lane, int &anti, int &ups)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    constexpr int RPL = Gm::RPL, G = Gm::G, H = Gm::H;
    const int gbase = lane & ~(G - 1);
    const int q = lane & (G - 1);
    const W nextA = __shfl_sync(0xffffffffu, A[0], gbase | ((q + 1) & (G - 1)));
    const W nextB = __shfl_sync(0xffffffffu, B[0], gbase | ((q + 1) & (G - 1)));
    anti = 0;
    ups = 0;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const bool odd = ((r0 + i) & 1) != 0;
        const W E = odd ? B[i] : A[i];
        const W Od = odd ? A[i] : B[i];
        anti += popc(E ^ Od) + popc(Od ^ rot_down<W, H>(E));
        const W An = (i == RPL - 1) ? nextA : A[i + 1];
        const W Bn = (i == RPL - 1) ? nextB : B[i + 1];
        anti += popc(A[i] ^ Bn) + popc(B[i] ^ An);
        ups += popc(A[i]) + popc(B[i]);
    }
}

// ------------------------------------------------------------------------------------
// Fused kernel: (INIT) generate or (!INIT) load each replica, theta sweeps with the
// Metropolis (!HB) or heatbath (HB) update, measure.
// ------------------------------------------------------------------------------------
template <int L, bool INIT, bool HB>
__global__ void __launch_bounds__(sweep_threads(L), sweep_min_blocks(L)) k_sweep(SweepArgs a)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    constexpr int N = Gm::N, G = Gm::G, RPW = Gm::RPW, RPL = Gm::RPL;
    extern __shared__ int sh_hist[];

    for (int k = threadIdx.x; k <= N; k += blockDim.x) sh_hist[k] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int q = lane & (G - 1);
    const int sub = lane / G;
    const int r0 = q * RPL;
    const long long R = INIT ? a.R_init : a.st->R_cur;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;

    unsigned int rk0[10], rk1[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        rk0[i] = a.k0 + (unsigned int)i * kPhiloxW0;
        rk1[i] = a.k1 + (unsigned int)i * kPhiloxW1;
    }
    const Accept<W> ac = make_accept<L>(a.T4, a.T8);
    if (!INIT && blockIdx.x == 0 && threadIdx.x == 0 && (a.T4 != a.st->T4 || a.T8 != a.st->T8))
        set_error(a.st, PA_ERR_NUMERIC);  // host and device thresholds disagree (never expected)

    // per-block exact sums: |M|, M^2, and the levels at the step start (0) and now (1):
    // k0, k0^2, k1, k1^2, k0 k1
    __shared__ unsigned long long sh_sum[7];
    if (threadIdx.x < 7) sh_sum[threadIdx.x] = 0;
    __syncthreads();
    W *spins = reinterpret_cast<W *>(a.spins);
    constexpr int TQ = SweepStyle<L>::TQ_LEN;  // per warp
    constexpr int kWarps = sweep_threads(L) / 32;
    __shared__ W tq_eq[kWarps * TQ], tq_a4[kWarps * TQ], tq_inv[HB ? kWarps * TQ : 1];
    __shared__ unsigned int tq_code[kWarps * TQ];
    const int wib = threadIdx.x >> 5;
    const TieQueue<W> tq{tq_eq + wib * TQ, tq_a4 + wib * TQ, HB ? tq_inv + wib * TQ : nullptr,
                         tq_code + wib * TQ};

    for (long long base = warp * RPW; base < R; base += nwarps * RPW) {
        const long long j = base + sub;
        const bool active = j < R;
        W A[RPL], B[RPL];
        W *rep = spins + (size_t)(active ? j : 0) * (2 * L);
        const unsigned int slot = (unsigned int)j + a.slot_base;  // global replica slot
        if (INIT) {
            init_rows<L>(slot, r0, a.k0, a.k1, A, B);
        } else {
            if (active) load_rows<L>(rep, r0, A, B);
            else {
#pragma unroll
                for (int i = 0; i < RPL; ++i) { A[i] = 0; B[i] = 0; }
            }
        }
        sweep_rows<L, HB>(A, B, r0, lane, slot, (unsigned int)base + a.slot_base, a.t0, a.theta, a.step, rk0, rk1, ac,
                          tq);
        int anti, ups;
        measure_rows<L>(A, B, r0, lane, anti, ups);
        anti = group_sum<G>(anti);
        ups = group_sum<G>(ups);
        // exact sums of this group of replicas: |M|, M^2, k0, k0^2, k1, k1^2, k0 k1
        unsigned long long v[7] = {0, 0, 0, 0, 0, 0, 0};
        int level = -1;
        if (active) {
            if (INIT || a.theta > 0) store_rows<L>(rep, r0, A, B);
            if (q == 0) {
                level = anti >> 1;
                const int M = 2 * ups - N;
                if (!INIT) {
                    // level at the start of this temperature step (right after resampling),
                    // kept in level_snap by the step's first call
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
                v[0] = (unsigned long long)(M < 0 ? -M : M);
                v[1] = (unsigned long long)((long long)M * M);
            }
        }
        constexpr int NSUM = INIT ? 2 : 7;
        if constexpr (RPW >= 8) {
            // many replicas per warp: reduce over the warp first, and count equal levels once
            const unsigned int grp = __match_any_sync(0xffffffffu, level);
            if (level >= 0 && lane == __ffs((int)grp) - 1) atomicAdd(&sh_hist[level], __popc(grp));
#pragma unroll
            for (int i = 0; i < NSUM; ++i)
#pragma unroll
                for (int o = 16; o >= G; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
            if (lane == 0)
#pragma unroll
                for (int i = 0; i < NSUM; ++i) atomicAdd(&sh_sum[i], v[i]);
        } else if (level >= 0) {
            atomicAdd(&sh_hist[level], 1);
#pragma unroll
            for (int i = 0; i < NSUM; ++i) atomicAdd(&sh_sum[i], v[i]);
        }
    }

    // one global atomic per block and sum
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
    __syncthreads();
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
        const int v = sh_hist[k];
        if (v) atomicAdd(&a.hist[k], v);
    }
}

template <int L, bool INIT, bool HB>
cudaError_t launch_sweep_t(const SweepArgs &a, int num_sms, cudaStream_t s)
{
    constexpr int N = Geo<L>::N;
    const size_t smem = (size_t)(N + 1) * sizeof(int);
    // the dynamic shared-memory limit is a per-device attribute: raised once per device; the
    // occupancy (the same on every device of one kind) is queried with it
    static PerDeviceOnce once;
    static int blocks_per_sm = 0;
    cudaError_t e = once([&] {
        cudaError_t r = cudaFuncSetAttribute(k_sweep<L, INIT, HB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        int b = 0;
        if (r == cudaSuccess)
            r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep<L, INIT, HB>, sweep_threads(L), smem);
        if (r == cudaSuccess) blocks_per_sm = b > 0 ? b : 1;
        return r;
    });
    if (e != cudaSuccess) return e;
    const long long R = a.R_bound;
    const long long groups = (R + Geo<L>::RPW - 1) / Geo<L>::RPW;  // warps needed
    constexpr int kWarps = sweep_threads(L) / 32;
    long long blocks = (groups + kWarps - 1) / kWarps;
    const long long cap = (long long)num_sms * blocks_per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_sweep<L, INIT, HB><<<(unsigned int)blocks, sweep_threads(L), smem, s>>>(a);
    return cudaGetLastError();
}


}  // namespace pa
