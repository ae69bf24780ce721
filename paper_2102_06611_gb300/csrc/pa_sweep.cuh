// pa_sweep.cuh -- step 1 (simple-sampling initialisation) and step 3 (theta checkerboard
// Metropolis sweeps) of population annealing (arXiv:2102.06611, Sec. II), each fused with
// the measurement of step 4 (energy level, magnetisation, level histogram, exact sums).
//
// One replica is held entirely in registers by G lanes of a warp (lane g owns RPL rows,
// two half-row words per row), so all theta sweeps run without touching memory: a replica
// is read once and written once per call.  Neighbouring rows owned by other lanes come in
// through warp shuffles.  The update of one colour of one row is bit-sliced over the whole
// half-row word: aligned-neighbour classes come from XNORs of the four neighbour words, and
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

// Minimum resident blocks of 256 threads per SM the sweep kernel is compiled for (caps its
// registers at 65536 / (256 * n)).
#ifndef PA_SWEEP_MIN_BLOCKS
#define PA_SWEEP_MIN_BLOCKS 2
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

__device__ __forceinline__ PhiloxC0 philox_c0_setup(unsigned int c1, unsigned int c2, unsigned int c3,
                                                    const unsigned int *rk0, const unsigned int *rk1)
{
    PhiloxC0 p;
    unsigned int h1, l1;
    mulhilo(kPhiloxM1, c2, h1, l1);
    p.u0 = h1 ^ c1 ^ rk0[0];
    p.u1 = l1;
    p.u2 = c3 ^ rk1[0];
    mulhilo(kPhiloxM0, p.u0, p.v_hi, p.v_lo);
    p.u1k = p.u1 ^ rk0[1];
    return p;
}

__device__ __forceinline__ uint4 philox_c0(unsigned int c0, const PhiloxC0 &p, const unsigned int *rk0,
                                           const unsigned int *rk1)
{
    unsigned int hi0, lo0;
    mulhilo(kPhiloxM0, c0, hi0, lo0);
    // round 1: (u0, u1, hi0 ^ c3 ^ k1, lo0); round 2 with the shared M0 * u0
    const unsigned int z2 = hi0 ^ p.u2, z3 = lo0;
    unsigned int h1, l1;
    mulhilo(kPhiloxM1, z2, h1, l1);
    uint4 c = make_uint4(h1 ^ p.u1k, l1, p.v_hi ^ z3 ^ rk1[1], p.v_lo);
#pragma unroll
    for (int i = 2; i < 10; ++i) {
        unsigned int h0, l0, h1, l1;
        mulhilo(kPhiloxM0, c.x, h0, l0);
        mulhilo(kPhiloxM1, c.z, h1, l1);
        c = make_uint4(h1 ^ c.y ^ rk0[i], l1, h0 ^ c.w ^ rk1[i], l0);
    }
    return c;
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

// Per-launch constants of the acceptance test.  T = floor(e^{-4 beta} 2^32) (class a = 3)
// or floor(e^{-8 beta} 2^32) (class a = 4), T in [0, 2^32]: m[k] = all ones iff bit 31 - k of
// T is set (top 8 bits as bit-plane masks), low = T mod 2^24, alw = all ones iff T = 2^32.
template <typename W>
struct Accept {
    W m4[8], m8[8];
    W alw4, alw8;
    unsigned int low4, low8;
};

template <typename W>
__device__ __forceinline__ Accept<W> make_accept(unsigned long long T4, unsigned long long T8)
{
    Accept<W> c;
    const bool all4 = T4 >= (1ull << 32), all8 = T8 >= (1ull << 32);
    const unsigned int t4 = all4 ? 0u : (unsigned int)T4, t8 = all8 ? 0u : (unsigned int)T8;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        c.m4[k] = ((t4 >> (31 - k)) & 1u) ? ~W(0) : W(0);
        c.m8[k] = ((t8 >> (31 - k)) & 1u) ? ~W(0) : W(0);
    }
    c.alw4 = all4 ? ~W(0) : W(0);
    c.alw8 = all8 ? ~W(0) : W(0);
    c.low4 = t4 & 0xFFFFFFu;
    c.low8 = t8 & 0xFFFFFFu;
    return c;
}

// One colour (compile-time Q) of one sweep over the rows a lane holds.
//
// Acceptance x < T is decided bit-serially over the 32 sites of a word at once: the top 8
// bits of every site's uniform x are 8 bit planes (bit j of plane k is bit 31 - k of site j's
// x), compared most significant first against the class threshold's bits; a site stays
// undecided only while its bits equal the threshold's, which after 8 planes happens with
// probability 2^-8, and only then is its low 24-bit part drawn.  Plane k of row r is word
// k mod 4 of Philox(ctr = (2 (nh r + h) + k / 4, slot, SWEEP << 28 | tag, i)) for the 32-site
// chunk h of the half-row (nh = chunks per half-row); the low part of site j is the low 24
// bits of word 0 of Philox(ctr = (64 r + j, slot, REFINE << 28 | tag, i)), tag = 2t + Q.
template <int L, int Q>
__device__ __forceinline__ void half_sweep(typename Geo<L>::W *A, typename Geo<L>::W *B, int r0,
                                           int lane, unsigned int slot, unsigned int tag,
                                           unsigned int step, const unsigned int *rk0,
                                           const unsigned int *rk1, unsigned int k0, unsigned int k1,
                                           const Accept<typename Geo<L>::W> &ac)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    constexpr int RPL = Gm::RPL, G = Gm::G, H = Gm::H;
    constexpr int NH = Gm::WIDE ? 2 : 1;  // 32-site chunks per half-row
    W *T = (Q == 0) ? A : B;          // words updated by this colour
    const W *O = (Q == 0) ? B : A;    // the other half of each row (read only here)

    // rows r0 - 1 and r0 + RPL come from the neighbouring lanes of the group
    const int gbase = lane & ~(G - 1);
    const int q = lane & (G - 1);
    const W from_up = __shfl_sync(0xffffffffu, O[RPL - 1], gbase | ((q - 1) & (G - 1)));
    const W from_down = __shfl_sync(0xffffffffu, O[0], gbase | ((q + 1) & (G - 1)));

    // the plane stream's calls differ only in c0 (rounds 1 and 2 partly shared)
    const PhiloxC0 pc = philox_c0_setup(slot, (kStreamSweep << 28) | tag, step, rk0, rk1);

    W lt[RPL], eq[RPL], a4[RPL], g3[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const int r = r0 + i;
        const W s = T[i];
        const W up = (i == 0) ? from_up : O[i - 1];
        const W dn = (i == RPL - 1) ? from_down : O[i + 1];
        const W h_a = O[i];
        // the updated half is the even-column half iff (r + Q) is even
        const bool even_half = ((r + Q) & 1) == 0;
        const W h_b = even_half ? rot_up<W, H>(O[i]) : rot_down<W, H>(O[i]);
        const W x1 = ~(s ^ up), x2 = ~(s ^ dn), x3 = ~(s ^ h_a), x4 = ~(s ^ h_b);
        const W all4 = x1 & x2 & x3 & x4 & half_mask<W, H>();
        const W ge3 = ((x1 & x2 & (x3 | x4)) | (x3 & x4 & (x1 | x2))) & half_mask<W, H>();
        const W eq3 = ge3 & ~all4;

        // bit planes of the top 8 bits of every site's uniform
        W plane[8];
        if constexpr (NH == 1) {
            const uint4 p0 = philox_c0((unsigned int)(2 * r), pc, rk0, rk1);
            const uint4 p1 = philox_c0((unsigned int)(2 * r + 1), pc, rk0, rk1);
            plane[0] = p0.x; plane[1] = p0.y; plane[2] = p0.z; plane[3] = p0.w;
            plane[4] = p1.x; plane[5] = p1.y; plane[6] = p1.z; plane[7] = p1.w;
        } else {
            const uint4 a0 = philox_c0((unsigned int)(4 * r), pc, rk0, rk1);
            const uint4 a1 = philox_c0((unsigned int)(4 * r + 1), pc, rk0, rk1);
            const uint4 b0 = philox_c0((unsigned int)(4 * r + 2), pc, rk0, rk1);
            const uint4 b1 = philox_c0((unsigned int)(4 * r + 3), pc, rk0, rk1);
            const unsigned int lo[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const unsigned int hi[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) plane[k] = (W)lo[k] | ((W)hi[k] << 32);
        }
        W l = (eq3 & ac.alw4) | (all4 & ac.alw8);   // decided: x < T
        W e = (eq3 & ~ac.alw4) | (all4 & ~ac.alw8); // undecided: top bits equal so far
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const W tm = (eq3 & ac.m4[k]) | (all4 & ac.m8[k]);  // threshold bit of each site
            l |= e & ~plane[k] & tm;
            e &= ~(plane[k] ^ tm);
        }
        lt[i] = l;
        eq[i] = e;
        a4[i] = all4;
        g3[i] = ge3;
    }

    // rare: the low 24 bits decide the sites whose top 8 bits equal the threshold's; one
    // loop over all rows of the lane keeps the warp's divergent iterations few
    W pending = 0;
#pragma unroll
    for (int i = 0; i < RPL; ++i) pending |= eq[i];
    while (pending) {
        int isel = 0;
        W w = 0, a4s = 0;
#pragma unroll
        for (int i = RPL - 1; i >= 0; --i)
            if (eq[i]) {
                isel = i;
                w = eq[i];
                a4s = a4[i];
            }
        const int j = Gm::WIDE ? __ffsll((long long)w) - 1 : __ffs((int)w) - 1;
        const uint4 xr = philox(make_uint4((unsigned int)(64 * (r0 + isel) + j), slot, (kStreamRefine << 28) | tag,
                                           step), k0, k1);
        const unsigned int thr = ((a4s >> j) & W(1)) ? ac.low8 : ac.low4;
        const W bit = W(1) << j;
        const W acc = ((xr.x & 0xFFFFFFu) < thr) ? bit : W(0);
        pending = 0;
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
            if (i == isel) {
                eq[i] &= ~bit;
                lt[i] |= acc;
            }
            pending |= eq[i];
        }
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i) T[i] ^= (~g3[i] | lt[i]) & half_mask<W, H>();
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

// Fused kernel: (INIT) generate or (!INIT) load each replica, theta sweeps, measure.

}  // namespace pa
