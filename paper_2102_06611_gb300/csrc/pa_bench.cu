// pa_bench.cu -- a measurement kernel, not a step of the method: Philox4x32-10 calls alone
// (Salmon, Moraes, Dror and Shaw, SC'11) with the sweep's round function (precomputed round
// keys, the 64-bit products as separate low and high multiplies) and, as in the sweep, calls
// that differ only in counter word 0; the four output words are XOR-reduced per thread so
// that nothing but the generator's arithmetic is timed.  Two calls give the 8 bit planes of 32
// Metropolis attempts, so 16 x the call rate is the rate at which the sweep could run if it did
// nothing but draw its random numbers.  Of the two ways to write these calls this is the
// faster alone (about 500 calls/ns on a GB300, the compiler hoisting the product that does not
// depend on word 0); the sweep's explicit sharing of rounds 1 and 2 (philox_c0, faster inside
// the sweep) runs at about 364 calls/ns here, so the rate reported is the higher ceiling.
#include "pa_sweep.cuh"

namespace pa {
namespace {

constexpr unsigned int kStreamBench = 15u;  // a counter stream no step of the method uses
constexpr int kBenchThreads = 256;

// out[t] = XOR over i < calls of the four words of Philox(ctr = (i, t, 15 << 28, 0)).
__global__ void __launch_bounds__(kBenchThreads) k_philox_xor(unsigned int k0, unsigned int k1, int calls,
                                                              int n_threads, unsigned int *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_threads) return;
    unsigned int rk0[10], rk1[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        rk0[i] = k0 + (unsigned int)i * kPhiloxW0;
        rk1[i] = k1 + (unsigned int)i * kPhiloxW1;
    }
    unsigned int acc = 0;
#pragma unroll 2
    for (int i = 0; i < calls; ++i) {
        const uint4 x = philox_rk(make_uint4((unsigned int)i, (unsigned int)t, kStreamBench << 28, 0u), rk0, rk1);
        acc ^= x.x ^ x.y ^ x.z ^ x.w;
    }
    out[t] = acc;
}

}  // namespace
}  // namespace pa

extern "C" pa_status pa_philox_xor(unsigned long long seed, int n_threads, int calls, unsigned int *out_dev,
                                   void *stream)
{
    if (n_threads < 1 || calls < 0 || !out_dev) return PA_ERR_INVALID_ARG;
    const unsigned int k0 = (unsigned int)(seed & 0xffffffffu), k1 = (unsigned int)(seed >> 32);
    const int blocks = (n_threads + pa::kBenchThreads - 1) / pa::kBenchThreads;
    pa::k_philox_xor<<<blocks, pa::kBenchThreads, 0, static_cast<cudaStream_t>(stream)>>>(k0, k1, calls, n_threads,
                                                                                        out_dev);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}
