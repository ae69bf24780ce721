// pa_sweep.cu -- step 1 (simple-sampling initialisation) and step 3 (theta checkerboard
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
// x < floor(e^{-8 beta} 2^32), with x a 32-bit Philox word.  Random word for the colour-q
// site with index j (column 2j + ((r + q) & 1)) of row r in sweep t of step i, slot s:
// lane (j & 3) of Philox(key = seed, ctr = (16 r + j / 4, s, SWEEP << 28 | (2t + q), i)).
#include "pa_common.cuh"
#include "pa_kernels.h"

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

// Philox4x32-10 with the first round's uniform half precomputed: u0 = hi(M1 c2) ^ c1 ^ k0,
// u1 = lo(M1 c2), u2 = c3 ^ k1; only c0 varies between calls.
__device__ __forceinline__ uint4 philox_c0(unsigned int c0, unsigned int u0, unsigned int u1,
                                           unsigned int u2, const unsigned int *rk0,
                                           const unsigned int *rk1)
{
    unsigned int hi0, lo0;
    mulhilo(kPhiloxM0, c0, hi0, lo0);
    uint4 c = make_uint4(u0, u1, hi0 ^ u2, lo0);
#pragma unroll
    for (int i = 1; i < 10; ++i) {
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

// One colour (compile-time Q) of one sweep over the rows a lane holds.
template <int L, int Q>
__device__ __forceinline__ void half_sweep(typename Geo<L>::W *A, typename Geo<L>::W *B, int r0,
                                           int lane, unsigned int slot, unsigned int tag,
                                           unsigned int step, const unsigned int *rk0,
                                           const unsigned int *rk1, unsigned int tm1_4,
                                           unsigned int tm1_8, typename Geo<L>::W nz4,
                                           typename Geo<L>::W nz8)
{
    using Gm = Geo<L>;
    using W = typename Gm::W;
    constexpr int RPL = Gm::RPL, G = Gm::G, H = Gm::H;
    constexpr int NGRP = (H + 3) / 4;
    W *T = (Q == 0) ? A : B;          // words updated by this colour
    const W *O = (Q == 0) ? B : A;    // the other half of each row (read only here)

    // rows r0 - 1 and r0 + RPL come from the neighbouring lanes of the group
    const int gbase = lane & ~(G - 1);
    const int q = lane & (G - 1);
    const W from_up = __shfl_sync(0xffffffffu, O[RPL - 1], gbase | ((q - 1) & (G - 1)));
    const W from_down = __shfl_sync(0xffffffffu, O[0], gbase | ((q + 1) & (G - 1)));

    // first Philox round: the c2 = tag product and the slot / step words are uniform here
    unsigned int h1, l1;
    mulhilo(kPhiloxM1, tag, h1, l1);
    const unsigned int u0 = h1 ^ slot ^ rk0[0];
    const unsigned int u1 = l1;
    const unsigned int u2 = step ^ rk1[0];

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
        const W all4 = x1 & x2 & x3 & x4;
        const W ge3 = (x1 & x2 & (x3 | x4)) | (x3 & x4 & (x1 | x2));
        const W eq3 = ge3 & ~all4;
        W acc3 = 0, acc4 = 0;
#pragma unroll
        for (int g = 0; g < NGRP; ++g) {
            const uint4 x = philox_c0((unsigned int)(16 * r + g), u0, u1, u2, rk0, rk1);
            const unsigned int xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = 4 * g + k;
                if (j < H) {
                    acc3 |= (W)(xs[k] <= tm1_4) << j;
                    acc4 |= (W)(xs[k] <= tm1_8) << j;
                }
            }
        }
        acc3 &= nz4;
        acc4 &= nz8;
        const W flip = (~ge3 | (eq3 & acc3) | (all4 & acc4)) & half_mask<W, H>();
        T[i] = s ^ flip;
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

// Fused kernel: (INIT) generate or (!INIT) load each replica, theta sweeps, measure.
template <int L, bool INIT>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a)
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
    const unsigned int tm1_4 = a.st->tm1_4, tm1_8 = a.st->tm1_8;
    const W nz4 = a.st->nz_4 ? ~W(0) : W(0);
    const W nz8 = a.st->nz_8 ? ~W(0) : W(0);

    unsigned long long s_abs = 0, s_m2 = 0;
    W *spins = reinterpret_cast<W *>(a.spins);

    for (long long base = warp * RPW; base < R; base += nwarps * RPW) {
        const long long j = base + sub;
        const bool active = j < R;
        W A[RPL], B[RPL];
        W *rep = spins + (size_t)(active ? j : 0) * (2 * L);
        if (INIT) {
            init_rows<L>((unsigned int)j, r0, a.k0, a.k1, A, B);
        } else {
            if (active) load_rows<L>(rep, r0, A, B);
            else {
#pragma unroll
                for (int i = 0; i < RPL; ++i) { A[i] = 0; B[i] = 0; }
            }
        }
#pragma unroll 1
        for (int t = 0; t < a.theta; ++t) {
            const unsigned int tag0 = (kStreamSweep << 28) | (unsigned int)(2 * (a.t0 + t));
            half_sweep<L, 0>(A, B, r0, lane, (unsigned int)j, tag0, a.step, rk0, rk1, tm1_4,
                             tm1_8, nz4, nz8);
            half_sweep<L, 1>(A, B, r0, lane, (unsigned int)j, tag0 | 1u, a.step, rk0, rk1, tm1_4,
                             tm1_8, nz4, nz8);
        }
        int anti, ups;
        measure_rows<L>(A, B, r0, lane, anti, ups);
        anti = group_sum<G>(anti);
        ups = group_sum<G>(ups);
        if (active) {
            if (INIT || a.theta > 0) store_rows<L>(rep, r0, A, B);
            if (q == 0) {
                const int level = anti >> 1;
                const int M = 2 * ups - N;
                a.level[j] = level;
                a.mag[j] = M;
                if (INIT) a.fam[j] = (int)j;
                atomicAdd(&sh_hist[level], 1);
                s_abs += (unsigned long long)(M < 0 ? -M : M);
                s_m2 += (unsigned long long)((long long)M * M);
            }
        }
    }

    // block reduction of the exact sums, then one global atomic per block
    s_abs = group_sum<32>(s_abs);
    s_m2 = group_sum<32>(s_m2);
    if (lane == 0 && (s_abs | s_m2)) {
        atomicAdd(&a.st->sum_absM, s_abs);
        atomicAdd(&a.st->sum_M2, s_m2);
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
        const int v = sh_hist[k];
        if (v) atomicAdd(&a.hist[k], v);
    }
}

template <int L, bool INIT>
static cudaError_t launch_sweep_t(const SweepArgs &a, int num_sms, cudaStream_t s)
{
    constexpr int N = Geo<L>::N;
    const size_t smem = (size_t)(N + 1) * sizeof(int);
    static int blocks_per_sm = 0;  // occupancy of this instantiation, queried once
    if (blocks_per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<L, INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep<L, INIT>, 256, smem);
        if (e != cudaSuccess) return e;
        blocks_per_sm = b > 0 ? b : 1;
    }
    const long long R = a.R_bound;
    const long long groups = (R + Geo<L>::RPW - 1) / Geo<L>::RPW;  // warps needed
    long long blocks = (groups + 7) / 8;
    const long long cap = (long long)num_sms * blocks_per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_sweep<L, INIT><<<(unsigned int)blocks, 256, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep(int L, bool init, const SweepArgs &a, int num_sms, cudaStream_t s)
{
#define PA_SWEEP_CASE(LL)                                                                      \
    case LL:                                                                                   \
        return init ? launch_sweep_t<LL, true>(a, num_sms, s) : launch_sweep_t<LL, false>(a, num_sms, s);
    switch (L) {
        PA_SWEEP_CASE(4)
        PA_SWEEP_CASE(8)
        PA_SWEEP_CASE(12)
        PA_SWEEP_CASE(16)
        PA_SWEEP_CASE(24)
        PA_SWEEP_CASE(32)
        PA_SWEEP_CASE(48)
        PA_SWEEP_CASE(64)
        PA_SWEEP_CASE(128)
        default:
            return cudaErrorInvalidValue;
    }
#undef PA_SWEEP_CASE
}

}  // namespace pa
