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
__global__ void __launch_bounds__(1024) k_features(FeatureArgs a)
{
    __shared__ double red[32][4];
    __shared__ double tot[4];
    const int N = a.L * a.L, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // block sums of NV values, valid in every thread: a shuffle tree in each warp, then one
    // over the 32 warp sums in warp 0 (binary64 work is slow here, so no serial loops)
    auto block_sums = [&](double *v, int nv) {
        for (int i = 0; i < nv; ++i)
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        if (lane == 0)
            for (int i = 0; i < nv; ++i) red[wid][i] = v[i];
        __syncthreads();
        if (wid == 0)
            for (int i = 0; i < nv; ++i) {
                double t = red[lane][i];
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == 0) tot[i] = t;
            }
        __syncthreads();
        for (int i = 0; i < nv; ++i) v[i] = tot[i];
        __syncthreads();  // red and tot are reused by the next call
    };
    // empty levels add exact zeros: skipping them leaves every sum unchanged
    double v1[2] = {0.0, 0.0};  // sum h, sum h E
    for (int k = tid; k <= N; k += 1024) {
        const int hk = a.hist[k];
        if (hk == 0) continue;
        const double h = (double)hk;
        v1[0] += h;
        v1[1] += h * (4.0 * k - 2.0 * N);
    }
    block_sums(v1, 2);
    const double R = v1[0], mean = v1[1] / R;
    double v2[4] = {0.0, 0.0, 0.0, 0.0};  // central sums of order 2, 3, 4; sum of squared family sizes
    for (int k = tid; k <= N; k += 1024) {
        const int hk = a.hist[k];
        if (hk == 0) continue;
        const double h = (double)hk;
        const double d = (4.0 * k - 2.0 * N) - mean;
        v2[0] += h * d * d;
        v2[1] += h * d * d * d;
        v2[2] += h * d * d * d * d;
    }
    for (int b = tid; b < kFamBlocks; b += 1024) v2[3] += (double)a.fampart[2 * b + 1];
    block_sums(v2, 4);
    const double var = v2[0] / R, m3 = v2[1] / R, m4 = v2[2] / R, size2 = v2[3];
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
            case 5: f = var > 0 ? m3 / pow(var, 1.5) : 0.0; break;
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
