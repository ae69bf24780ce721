// pa_common.cuh -- device-side building blocks shared by the library's translation units:
// lattice geometry of the packed layout, Philox4x32-10, the deterministic binary64 exp,
// and the device state block kept in the caller's workspace.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pa.h"

// Rows of a replica held by one lane in the sweep kernel (tuning knobs; lanes per replica =
// L / rows, a power of two <= 32).
#ifndef PA_RPL_16
#define PA_RPL_16 16
#endif
#ifndef PA_RPL_24
#define PA_RPL_24 12
#endif
#ifndef PA_RPL_32
#define PA_RPL_32 8
#endif
#ifndef PA_RPL_48
#define PA_RPL_48 6
#endif
#ifndef PA_RPL_64
#define PA_RPL_64 4
#endif
#ifndef PA_RPL_128
#define PA_RPL_128 4
#endif

namespace pa {

// ------------------------------------------------------------------------------------
// Packed spin layout.  Row r of a replica is stored as two half-rows: half 0 holds the
// spins at even columns 2j (bit j), half 1 those at odd columns 2j + 1 (bit j); bit set
// = spin +1.  A half-row of H = L/2 bits is one uint32 (L <= 64) or one uint64 (L = 128).
// Rows follow each other; a replica is L * 2 half-row words, contiguous.
//
// In the checkerboard update the sites of colour q = (r + c) mod 2 in row r are exactly
// half (r + q) mod 2 of that row, so one colour of one row is one whole word.
//
// A replica is handled by G lanes of a warp; lane g holds rows g*RPL .. g*RPL + RPL - 1.
//
// Random bit planes of the Metropolis test come per 32-site chunk of one colour: the sites
// of colour q are numbered n = r H' + p (p = c / 2, rows padded to H', the smallest power of
// two >= H) and chunk n / 32 holds bit n mod 32.  For L >= 48 a chunk lies within one row;
// for smaller L it spans P = 32 / H' rows (all L rows when L = 4), and the sweep kernel
// packs the P rows of a chunk into one register word ("packed" sizes).
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr int rows_per_lane(int L)
{
    return L == 4 ? 4 : L == 8 ? 8 : L == 12 ? 12 : L == 16 ? PA_RPL_16 : L == 20 ? 10 : L == 24 ? PA_RPL_24
           : L == 32 ? PA_RPL_32 : L == 40 ? 5 : L == 48 ? PA_RPL_48 : L == 64 ? PA_RPL_64 : L == 80 ? 5
           : L == 96 ? 6 : PA_RPL_128;
}

__host__ __device__ constexpr int padded_half(int L)
{
    int h = 1;
    while (h < L / 2) h *= 2;
    return h;
}

template <int L_>
struct Geo {
    static constexpr int L = L_;
    static constexpr int N = L * L;
    static constexpr int H = L / 2;                      // sites per half-row
    static constexpr bool WIDE = (H > 32);
    using W = typename std::conditional<WIDE, unsigned long long, unsigned int>::type;
    static constexpr int RPL = rows_per_lane(L);
    static constexpr int G = L / RPL;                    // lanes per replica (power of 2)
    static constexpr int RPW = 32 / G;                   // replicas per warp
    static constexpr int WORD_BYTES = WIDE ? 8 : 4;
    static constexpr int BYTES = L * 2 * WORD_BYTES;     // bytes per replica
    static constexpr int LANE_WORDS = 2 * RPL;           // half-row words held per lane
    static constexpr int HP = padded_half(L);            // H' (row pitch of the chunk numbering)
    static constexpr bool PACK = HP < 32;                // chunks span several rows
    static constexpr int P = PACK ? (32 / HP < L ? 32 / HP : L) : 1;  // rows per chunk
    static constexpr int CB = P * HP;                    // bits of a packed chunk word (32, or 8 at L = 4)
    static constexpr int C = RPL / P;                    // packed chunks per lane
    static_assert(L % RPL == 0, "rows per lane must divide L");
    static_assert((G & (G - 1)) == 0 && G <= 32 && G >= 1, "lanes per replica");
    static_assert(!PACK || (RPL % P == 0 && P % 2 == 0 && RPL % 2 == 0), "whole chunks of even rows per lane");
};

__host__ __device__ constexpr int bytes_per_replica(int L) { return L * 2 * (L / 2 > 32 ? 8 : 4); }

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies; the key is advanced by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------
constexpr unsigned int kPhiloxM0 = 0xD2511F53u;
constexpr unsigned int kPhiloxM1 = 0xCD9E8D57u;
constexpr unsigned int kPhiloxW0 = 0x9E3779B9u;
constexpr unsigned int kPhiloxW1 = 0xBB67AE85u;

enum : unsigned int {
    kStreamInit = 0u,
    kStreamSweep = 1u,
    kStreamResample = 2u,
    kStreamPoisson = 3u,
    kStreamRefine = 4u,
    kStreamMultinomial = 5u
};

// The 64-bit product of a Philox round as two separate multiplies (low word, high word) or
// as one widening multiply: the same values; the split form is measured 1-2 % faster in the
// sweep kernels of L >= 32 and 1-2 % slower below.
#ifndef PA_MULHI_SPLIT
#define PA_MULHI_SPLIT 1
#endif
template <bool SPLIT = (PA_MULHI_SPLIT != 0)>
__device__ __forceinline__ void mulhilo(unsigned int a, unsigned int b, unsigned int &hi, unsigned int &lo)
{
    if constexpr (SPLIT) {
        lo = a * b;
        hi = __umulhi(a, b);
    } else {
        unsigned long long p = (unsigned long long)a * (unsigned long long)b;
        hi = (unsigned int)(p >> 32);
        lo = (unsigned int)p;
    }
}

__device__ __forceinline__ uint4 philox(uint4 c, unsigned int k0, unsigned int k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        unsigned int hi0, lo0, hi1, lo1;
        mulhilo(kPhiloxM0, c.x, hi0, lo0);
        mulhilo(kPhiloxM1, c.z, hi1, lo1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// ------------------------------------------------------------------------------------
// Deterministic binary64 exp: Cody-Waite reduction x = k ln2 + r (ln2 = LN2_HI + LN2_LO,
// LN2_HI has 32 significant bits so k * LN2_HI is exact), then sum_{n<=13} r^n/n! in
// Horner form.  Every operation is an explicitly rounded binary64 intrinsic (no FMA
// contraction), so the value is a fixed function of x on every device.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double det_exp(double x)
{
    if (x != x) return x;
    if (x > 709.5) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -745.5) return 0.0;
    const double kLn2Hi = 0x1.62e42feep-1;
    const double kLn2Lo = 0x1.a39ef35793c76p-33;
    const double kInvLn2 = 0x1.71547652b82fep+0;
    double k = rint(__dmul_rn(x, kInvLn2));
    double r = __dadd_rn(__dadd_rn(x, -__dmul_rn(k, kLn2Hi)), -__dmul_rn(k, kLn2Lo));
    double p = 1.0 / 6227020800.0;
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 479001600.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 39916800.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 3628800.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 362880.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 40320.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 5040.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 720.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 120.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 24.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0 / 6.0);
    p = __dadd_rn(__dmul_rn(p, r), 0.5);
    p = __dadd_rn(__dmul_rn(p, r), 1.0);
    p = __dadd_rn(__dmul_rn(p, r), 1.0);
    return ldexp(p, (int)k);
}

// floor(exp(-y) 2^32) as a 64-bit integer in [0, 2^32].
__device__ __forceinline__ unsigned long long metropolis_threshold(double y)
{
    double p = det_exp(-y);
    return (unsigned long long)floor(__dmul_rn(p, 4294967296.0));
}

// floor(2^32 / (1 + exp(y))): the heatbath thresholds T_3 (y = 4 beta) and T_4 (y = 8 beta).
__device__ __forceinline__ unsigned long long heatbath_threshold(double y)
{
    double p = __ddiv_rn(1.0, __dadd_rn(1.0, det_exp(y)));
    return (unsigned long long)floor(__dmul_rn(p, 4294967296.0));
}

// ------------------------------------------------------------------------------------
// Device state block (first bytes of the workspace).
// ------------------------------------------------------------------------------------
struct DevState {
    long long R_cur;          // current population size R_i
    long long R_prev;         // population size before the last resampling R_{i-1}
    double lnQ;               // ln Q_i of the last resampling
    double sum_lnQ;           // running sum_k ln Q_k
    double S;                 // sum_k h_k w_k of the last resampling
    int kmin;                 // lowest occupied level of the last resampling
    int error;                // sticky pa_status bits (first error wins)
    // Metropolis thresholds at the current beta, floor(e^{-4 beta} 2^32) and
    // floor(e^{-8 beta} 2^32) in [0, 2^32]: a 32-bit uniform x is accepted iff x < T
    unsigned long long T4, T8;
    // exact integer sums of the current population (filled by measurement)
    unsigned long long sum_absM;
    unsigned long long sum_M2;
    long long fam_count;
    long long fam_size2;
    // result of the last schedule proposal
    double beta_next;
    double alpha_next;
    double dbeta_prop;        // learned proposal (before the overlap check)
    int theta_prop;
    int source_next;          // PA_SCHED_* of beta_next
    float y_prop[2];          // raw network outputs of the proposal
    // sums over replicas of the energy level at the start of the temperature step (k0) and
    // after the last sweep call (k1): sum k0, k0^2, k1, k1^2, k0 k1 (exact)
    long long c0, c00, c1, c11, c01;
    int theta;
    int update;               // pa_update_kind of the run (selects the thresholds below)
    unsigned long long mn_total;  // multinomial resampling: sum of the integer parent weights
    double sum_lnR;           // sum_k ln(R_{k-1} / R) over the resamplings so far
    long long R_glob;         // sharded population: the whole population's size (0 otherwise)
    // multinomial resampling of a sharded population: the integer weight sum of the parents of
    // the shards before this one (0 for a population held whole)
    unsigned long long mn_base;
};

// Block-wide exclusive prefix sum (every thread gets its prefix; *total the block sum) and
// block-wide sum (valid in thread 0).  Every thread of the block must call them.
template <typename T, int THREADS>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total)
{
    __shared__ T warp_tot[THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T t = lane < THREADS / 32 ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < THREADS / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    const T before = wid > 0 ? warp_tot[wid - 1] : T(0);
    *total = warp_tot[THREADS / 32 - 1];
    __syncthreads();
    return before + x - v;
}

template <typename T, int THREADS>
__device__ __forceinline__ T block_sum(T v)
{
    __shared__ T part[THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[wid] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < THREADS / 32; ++i) t += part[i];
    __syncthreads();
    return t;  // valid in thread 0
}

__device__ __forceinline__ void set_error(DevState *st, int code)
{
    atomicCAS(&st->error, 0, code);
}

// Warp-level reductions over aligned groups of G lanes.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace pa
