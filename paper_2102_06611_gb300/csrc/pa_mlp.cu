// pa_mlp.cu -- the learned temperature schedule: population features, a small MLP
// (12 -> 64 -> 64 -> 64 tanh -> 2) with bfloat16 parameters and float32 accumulation, its
// batched training kernels (forward, backward, Adam), and the proposal step that feeds the
// network's (dbeta, theta) through the histogram-overlap check of the step search (pa_schedule.cu).
//
// The paper has no learned schedule; it names self-adaptive steps (Sec. II), the overlap
// guideline alpha > 0.7 and an adaptive theta (Sec. X).  The network only proposes; every
// accepted step still satisfies the overlap floor, and the schedule actually used is logged
// so that the method can be replayed exactly.
#include <cmath>

#include <cuda_bf16.h>

#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {

// parameter offsets in the flat layout W1 [64x12], b1, W2 [64x64], b2, W3 [64x64], b3, W4 [2x64], b4
constexpr int kIn = 12, kHid = 64, kOut = 2;
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid * kHid, oW4 = oB3 + kHid, oB4 = oW4 + kOut * kHid, kParams = oB4 + kOut;
static_assert(kParams == 9282, "parameter count");
constexpr int kActs = 3 * kHid;          // a1, a2, a3 per sample
constexpr int kDeltas = 3 * kHid + kOut; // g1, g2, g3, g4 per sample

__device__ __forceinline__ float bf(const unsigned short *p, int i)
{
    return __uint_as_float((unsigned int)p[i] << 16);
}

// ------------------------------------------------------------------------------ forward
// One sample per 64 threads; thread j computes hidden unit j of each layer in turn.
__device__ __forceinline__ void mlp_forward_sample(const unsigned short *P, const float *x, float *a1, float *a2,
                                                   float *a3, float *y, int j)
{
    float s = bf(P, oB1 + j);
#pragma unroll
    for (int i = 0; i < kIn; ++i) s = fmaf(bf(P, oW1 + j * kIn + i), x[i], s);
    a1[j] = tanhf(s);
    __syncthreads();
    s = bf(P, oB2 + j);
    for (int i = 0; i < kHid; ++i) s = fmaf(bf(P, oW2 + j * kHid + i), a1[i], s);
    a2[j] = tanhf(s);
    __syncthreads();
    s = bf(P, oB3 + j);
    for (int i = 0; i < kHid; ++i) s = fmaf(bf(P, oW3 + j * kHid + i), a2[i], s);
    a3[j] = tanhf(s);
    __syncthreads();
    if (j < kOut) {
        s = bf(P, oB4 + j);
        for (int i = 0; i < kHid; ++i) s = fmaf(bf(P, oW4 + j * kHid + i), a3[i], s);
        y[j] = s;
    }
    __syncthreads();
}

constexpr int kSamplesPerBlock = 4;

__global__ void __launch_bounds__(kHid * kSamplesPerBlock) k_mlp_forward(const unsigned short *P, const float *x,
                                                                          int B, float *y, float *act)
{
    __shared__ float sx[kSamplesPerBlock][kIn];
    __shared__ float sa[kSamplesPerBlock][kActs];
    __shared__ float sy[kSamplesPerBlock][kOut];
    const int sub = threadIdx.x / kHid, j = threadIdx.x % kHid;
    const int b = blockIdx.x * kSamplesPerBlock + sub;
    const bool live = b < B;
    if (j < kIn) sx[sub][j] = live ? x[(size_t)b * kIn + j] : 0.f;
    __syncthreads();
    mlp_forward_sample(P, sx[sub], sa[sub], sa[sub] + kHid, sa[sub] + 2 * kHid, sy[sub], j);
    if (live) {
        if (act)
            for (int k = j; k < kActs; k += kHid) act[(size_t)b * kActs + k] = sa[sub][k];
        if (j < kOut) y[(size_t)b * kOut + j] = sy[sub][j];
    }
}

// ------------------------------------------------------------------------------ backward
// Per-sample deltas of L = 1/(2B) sum (y - t)^2: g4 = (y - t)/B, g3 = (g4 W4) * (1 - a3^2),
// g2 = (g3 W3) * (1 - a2^2), g1 = (g2 W2) * (1 - a1^2).
__global__ void __launch_bounds__(kHid * kSamplesPerBlock) k_mlp_deltas(const unsigned short *P, const float *t,
                                                                         int B, const float *act, const float *y,
                                                                         float *delta)
{
    __shared__ float sg[kSamplesPerBlock][kDeltas];
    const int sub = threadIdx.x / kHid, j = threadIdx.x % kHid;
    const int b = blockIdx.x * kSamplesPerBlock + sub;
    const bool live = b < B;
    const float invB = 1.0f / (float)B;
    float *g1 = sg[sub], *g2 = g1 + kHid, *g3 = g2 + kHid, *g4 = g3 + kHid;
    if (j < kOut) g4[j] = live ? (y[(size_t)b * kOut + j] - t[(size_t)b * kOut + j]) * invB : 0.f;
    __syncthreads();
    const float *a = live ? act + (size_t)b * kActs : nullptr;
    float s = 0.f;
    for (int o = 0; o < kOut; ++o) s = fmaf(g4[o], bf(P, oW4 + o * kHid + j), s);
    const float a3 = live ? a[2 * kHid + j] : 0.f;
    g3[j] = s * (1.f - a3 * a3);
    __syncthreads();
    s = 0.f;
    for (int k = 0; k < kHid; ++k) s = fmaf(g3[k], bf(P, oW3 + k * kHid + j), s);
    const float a2 = live ? a[kHid + j] : 0.f;
    g2[j] = s * (1.f - a2 * a2);
    __syncthreads();
    s = 0.f;
    for (int k = 0; k < kHid; ++k) s = fmaf(g2[k], bf(P, oW2 + k * kHid + j), s);
    const float a1 = live ? a[j] : 0.f;
    g1[j] = s * (1.f - a1 * a1);
    __syncthreads();
    if (live)
        for (int k = j; k < kDeltas; k += kHid) delta[(size_t)b * kDeltas + k] = sg[sub][k];
}

// Weight gradients: one thread per parameter, summing over the batch in sample order.
__global__ void k_mlp_wgrad(const float *x, int B, const float *act, const float *delta, float *grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    // which layer, which output unit (row) and which input (column, -1 for a bias)
    int d_off, row, col, in_kind;  // in_kind: 0 = x, 1 = a1, 2 = a2, 3 = a3, -1 = bias
    if (p < oB1) { d_off = 0; row = (p - oW1) / kIn; col = (p - oW1) % kIn; in_kind = 0; }
    else if (p < oW2) { d_off = 0; row = p - oB1; col = 0; in_kind = -1; }
    else if (p < oB2) { d_off = kHid; row = (p - oW2) / kHid; col = (p - oW2) % kHid; in_kind = 1; }
    else if (p < oW3) { d_off = kHid; row = p - oB2; col = 0; in_kind = -1; }
    else if (p < oB3) { d_off = 2 * kHid; row = (p - oW3) / kHid; col = (p - oW3) % kHid; in_kind = 2; }
    else if (p < oW4) { d_off = 2 * kHid; row = p - oB3; col = 0; in_kind = -1; }
    else if (p < oB4) { d_off = 3 * kHid; row = (p - oW4) / kHid; col = (p - oW4) % kHid; in_kind = 3; }
    else { d_off = 3 * kHid; row = p - oB4; col = 0; in_kind = -1; }
    float s = 0.f;
    for (int b = 0; b < B; ++b) {
        const float g = delta[(size_t)b * kDeltas + d_off + row];
        float in;
        if (in_kind < 0) in = 1.f;
        else if (in_kind == 0) in = x[(size_t)b * kIn + col];
        else in = act[(size_t)b * kActs + (in_kind - 1) * kHid + col];
        s = fmaf(g, in, s);
    }
    grad[p] = s;
}

__global__ void k_mlp_adam(float *master, float *m, float *v, const float *g, int step, float lr, float b1, float b2,
                           float eps, unsigned short *P)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float mi = b1 * m[p] + (1.f - b1) * g[p];
    const float vi = b2 * v[p] + (1.f - b2) * g[p] * g[p];
    m[p] = mi;
    v[p] = vi;
    const float mh = mi / (1.f - powf(b1, (float)step));
    const float vh = vi / (1.f - powf(b2, (float)step));
    const float w = master[p] - lr * mh / (sqrtf(vh) + eps);
    master[p] = w;
    P[p] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

__global__ void k_mlp_round(const float *master, unsigned short *P)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kParams) P[p] = __bfloat16_as_ushort(__float2bfloat16_rn(master[p]));
}

// ------------------------------------------------------------------------------ features
// The 12 inputs of the network from the current population, in binary64, then float32:
// beta, ln L, ln R, <E>/N, ln(Var(E)/N + 1e-12), skewness, excess kurtosis, dbeta_prev L,
// theta_prev / theta0, alpha_prev, ln(rho_t)/ln(R) (rho_t = sum of squared family sizes / R),
// fraction of parents with zero copies in the last resampling.
// A 128-bit two's-complement integer as two 64-bit words (exact sums of high powers).
struct I128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ I128 i128_add(I128 x, I128 y)
{
    I128 r;
    r.lo = x.lo + y.lo;
    r.hi = x.hi + y.hi + (r.lo < x.lo ? 1ull : 0ull);
    return r;
}
__device__ __forceinline__ I128 i128_from_prod(long long p, long long q)  // p * q, |p q| < 2^126
{
    const bool neg = (p < 0) != (q < 0);
    const unsigned long long up = (unsigned long long)(p < 0 ? -p : p), uq = (unsigned long long)(q < 0 ? -q : q);
    I128 r{up * uq, __umul64hi(up, uq)};
    if (neg) {  // two's complement
        r.lo = ~r.lo + 1ull;
        r.hi = ~r.hi + (r.lo == 0ull ? 1ull : 0ull);
    }
    return r;
}
__device__ __forceinline__ double i128_to_double(I128 x)
{
    const bool neg = (long long)x.hi < 0;
    if (neg) {
        x.lo = ~x.lo + 1ull;
        x.hi = ~x.hi + (x.lo == 0ull ? 1ull : 0ull);
    }
    const double v = __dadd_rn(__dmul_rn((double)x.hi, 18446744073709551616.0), (double)x.lo);
    return neg ? -v : v;
}
__device__ __forceinline__ I128 i128_shfl_xor(I128 x, int o)
{
    return I128{__shfl_xor_sync(0xffffffffu, x.lo, o), __shfl_xor_sync(0xffffffffu, x.hi, o)};
}

// The moments come from exact integer sums over the occupied levels (this GPU's binary64
// pipe is narrow, so the per-level work stays on the integer pipes): with the level index k,
// h_k replicas and d = k - k_ref about the rounded mean level k_ref, the sums of h d^p for
// p = 0 .. 4 are exact (128 bits for p = 3, 4), and the central moments of E = 4 k - 2 N
// follow in binary64 from them.  The binary64 features then take one warp each.
__global__ void __launch_bounds__(1024) k_features(FeatureArgs a)
{
    constexpr int kW = 1024 / 32;
    __shared__ long long sh_a[kW][2];
    __shared__ long long sh_b[kW][3];
    __shared__ I128 sh_c[kW][2];
    __shared__ long long sh_kref;
    __shared__ double sh_m[5];  // R, <E>, var, m3, m4
    __shared__ double sh_size2;
    const int N = a.L * a.L, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    // pass 1: sum h, sum h k (exact) -> the rounded mean level
    long long s0 = 0, s1 = 0;
    for (int k = tid; k <= N; k += 1024) {
        const long long h = a.hist[k];
        s0 += h;
        s1 += h * k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
        sh_a[wid][0] = s0;
        sh_a[wid][1] = s1;
    }
    __syncthreads();
    if (tid == 0) {
        long long t0 = 0, t1 = 0;
        for (int w = 0; w < kW; ++w) {
            t0 += sh_a[w][0];
            t1 += sh_a[w][1];
        }
        sh_a[0][0] = t0;
        sh_kref = t0 > 0 ? (t1 + t0 / 2) / t0 : 0;
    }
    __syncthreads();
    const long long R_int = sh_a[0][0], kref = sh_kref;

    // pass 2: sum h d, h d^2 (64 bits), h d^3, h d^4 (128 bits), sum of squared family sizes
    long long p1 = 0, p2 = 0, f2 = 0;
    I128 p3{0, 0}, p4{0, 0};
    for (int k = tid; k <= N; k += 1024) {
        const long long h = a.hist[k];
        if (h == 0) continue;
        const long long d = (long long)k - kref, hd2 = h * d * d;
        p1 += h * d;
        p2 += hd2;
        p3 = i128_add(p3, i128_from_prod(hd2, d));
        p4 = i128_add(p4, i128_from_prod(hd2, d * d));
    }
    for (int b = tid; b < kFamBlocks; b += 1024) f2 += a.fampart[2 * b + 1];
    for (int o = 16; o > 0; o >>= 1) {
        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
        p2 += __shfl_xor_sync(0xffffffffu, p2, o);
        f2 += __shfl_xor_sync(0xffffffffu, f2, o);
        p3 = i128_add(p3, i128_shfl_xor(p3, o));
        p4 = i128_add(p4, i128_shfl_xor(p4, o));
    }
    if (lane == 0) {
        sh_b[wid][0] = p1;
        sh_b[wid][1] = p2;
        sh_b[wid][2] = f2;
        sh_c[wid][0] = p3;
        sh_c[wid][1] = p4;
    }
    __syncthreads();
    if (tid == 0) {
        long long t1 = 0, t2 = 0, tf = 0;
        I128 t3{0, 0}, t4{0, 0};
        for (int w = 0; w < kW; ++w) {
            t1 += sh_b[w][0];
            t2 += sh_b[w][1];
            tf += sh_b[w][2];
            t3 = i128_add(t3, sh_c[w][0]);
            t4 = i128_add(t4, sh_c[w][1]);
        }
        // central moments in level units from the raw ones about k_ref, then of E = 4 k - 2 N
        const double R = (double)R_int;
        const double mu = (double)t1 / R, r2 = (double)t2 / R, r3 = i128_to_double(t3) / R,
                     r4 = i128_to_double(t4) / R;
        const double c2 = r2 - mu * mu;
        const double c3 = r3 - 3.0 * mu * r2 + 2.0 * mu * mu * mu;
        const double c4 = r4 - 4.0 * mu * r3 + 6.0 * mu * mu * r2 - 3.0 * mu * mu * mu * mu;
        sh_m[0] = R;
        sh_m[1] = 4.0 * ((double)kref + mu) - 2.0 * N;
        sh_m[2] = 16.0 * c2;
        sh_m[3] = 64.0 * c3;
        sh_m[4] = 256.0 * c4;
        sh_size2 = (double)tf;
    }
    __syncthreads();
    const double R = sh_m[0], mean = sh_m[1], var = sh_m[2], m3 = sh_m[3], m4 = sh_m[4], size2 = sh_size2;
    // one feature per warp (lane 0), so that the binary64 logarithms and powers run side by side
    if (lane == 0 && wid < kIn) {
        const long long R_prev = a.st->R_prev;
        double f = 0.0;
        switch (wid) {
            case 0: f = a.beta; break;
            case 1: f = log((double)a.L); break;
            case 2: f = log(R); break;
            case 3: f = mean / N; break;
            case 4: f = log(var / N + 1e-12); break;
            case 5: f = var > 0 ? m3 / (var * sqrt(var)) : 0.0; break;
            case 6: f = var > 0 ? m4 / (var * var) - 3.0 : 0.0; break;
            case 7: f = a.dbeta_prev * a.L; break;
            case 8: f = a.theta_ratio_prev; break;
            case 9: f = a.alpha_prev; break;
            case 10: {
                const double lnR = log(R);
                f = lnR > 0 ? log(size2 / R) / lnR : 0.0;
                break;
            }
            default: f = R_prev > 0 ? (double)*a.zeros / (double)R_prev : 0.0; break;  // exact below 2^53
        }
        a.raw[wid] = (float)f;
        a.x[wid] = a.norm ? ((float)f - a.norm[wid]) / a.norm[kIn + wid] : (float)f;
    }
}

// One network evaluation for the proposal: (dbeta, theta) from the de-standardised outputs
// y0 = ln(dbeta sigma_E) (the overlap of nearby energy distributions depends mainly on
// dbeta times the energy width sigma_E, so this target carries over between lattice sizes)
// and y1 = ln(theta); sigma_E^2 = N exp(raw feature 4); clamped to dbeta in (0, dbeta_max],
// theta in [1, theta_max].
__global__ void __launch_bounds__(kHid) k_mlp_propose(const unsigned short *P, const float *norm, const float *raw,
                                                      const float *x, int L, double dbeta_max, int theta_max,
                                                      DevState *st)
{
    __shared__ float sa[kActs];
    __shared__ float sy[kOut];
    const int j = threadIdx.x;
    mlp_forward_sample(P, x, sa, sa + kHid, sa + 2 * kHid, sy, j);
    if (j == 0) {
        const float y0 = sy[0] * norm[2 * kIn + kOut + 0] + norm[2 * kIn + 0];
        const float y1 = sy[1] * norm[2 * kIn + kOut + 1] + norm[2 * kIn + 1];
        const double sigma_E = sqrt((double)L * (double)L * exp((double)raw[4]));
        double dbeta = exp((double)y0) / sigma_E;
        if (!(dbeta > 0.0)) dbeta = 1e-12;
        if (dbeta > dbeta_max) dbeta = dbeta_max;
        double th = rint(exp((double)y1));
        if (!(th >= 1.0)) th = 1.0;
        if (th > (double)theta_max) th = (double)theta_max;
        st->dbeta_prop = dbeta;
        st->theta_prop = (int)th;
        st->y_prop[0] = sy[0];
        st->y_prop[1] = sy[1];
    }
}

// Parents with zero copies in the last resampling, over many blocks (one block reading every
// copy number took ~0.1 ms at R = 2e5): an exact integer count.
__global__ void __launch_bounds__(256) k_count_zeros(const DevState *st, const int *counts, unsigned long long *out)
{
    const long long Rp = st->R_prev;
    unsigned long long z = 0;
    for (long long j = (long long)blockIdx.x * 256 + threadIdx.x; j < Rp; j += (long long)gridDim.x * 256)
        z += counts[j] == 0;
    z = block_sum<unsigned long long, 256>(z);
    if (threadIdx.x == 0 && z) atomicAdd(out, z);
}

cudaError_t launch_features(const FeatureArgs &a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.zeros, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const long long want = (a.capacity + 1023) / 1024;
    const unsigned int blocks = (unsigned int)(want < 1 ? 1 : (want > 608 ? 608 : want));
    k_count_zeros<<<blocks, 256, 0, s>>>(a.st, a.counts, a.zeros);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_features<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_propose(const unsigned short *P, const float *norm, const float *raw, const float *x, int L,
                               double dbeta_max, int theta_max, DevState *st, cudaStream_t s)
{
    k_mlp_propose<<<1, kHid, 0, s>>>(P, norm, raw, x, L, dbeta_max, theta_max, st);
    return cudaGetLastError();
}

}  // namespace pa

// ------------------------------------------------------------------------------ C ABI
extern "C" {

size_t pa_mlp_param_count(void) { return (size_t)pa::kParams; }

pa_status pa_mlp_forward(const unsigned short *params_bf16, const float *x, int batch, float *y, float *act,
                         void *stream)
{
    if (!params_bf16 || !x || !y || batch < 1) return PA_ERR_INVALID_ARG;
    const unsigned int blocks = (unsigned int)((batch + pa::kSamplesPerBlock - 1) / pa::kSamplesPerBlock);
    pa::k_mlp_forward<<<blocks, pa::kHid * pa::kSamplesPerBlock, 0, static_cast<cudaStream_t>(stream)>>>(
        params_bf16, x, batch, y, act);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_mlp_backward(const unsigned short *params_bf16, const float *x, const float *t, int batch,
                          const float *act, const float *y, float *delta, float *grad, void *stream)
{
    if (!params_bf16 || !x || !t || !act || !y || !delta || !grad || batch < 1) return PA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned int blocks = (unsigned int)((batch + pa::kSamplesPerBlock - 1) / pa::kSamplesPerBlock);
    pa::k_mlp_deltas<<<blocks, pa::kHid * pa::kSamplesPerBlock, 0, s>>>(params_bf16, t, batch, act, y, delta);
    if (cudaGetLastError() != cudaSuccess) return PA_ERR_CUDA;
    pa::k_mlp_wgrad<<<(pa::kParams + 255) / 256, 256, 0, s>>>(x, batch, act, delta, grad);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_mlp_adam(float *master, float *m, float *v, const float *grad, int step, float lr, float beta1,
                      float beta2, float eps, unsigned short *params_bf16, void *stream)
{
    if (!master || !m || !v || !grad || !params_bf16 || step < 1) return PA_ERR_INVALID_ARG;
    pa::k_mlp_adam<<<(pa::kParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        master, m, v, grad, step, lr, beta1, beta2, eps, params_bf16);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_mlp_round(const float *master, unsigned short *params_bf16, void *stream)
{
    if (!master || !params_bf16) return PA_ERR_INVALID_ARG;
    pa::k_mlp_round<<<(pa::kParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(master, params_bf16);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

}  // extern "C"
