// pa_analysis.cu -- population analysis of population annealing (arXiv:2102.06611): blocked
// and jackknife errors of the mean over the tree-ordered population and the effective
// population size R_eff (Sec. IV, Eqs. neff, blocks, blocked_variance, jackknife-blocks,
// jackknife-variance), and the family entropy S_f with rho_s = R / exp(S_f) (Sec. V,
// Eq. rhos); and the weighted average of independent runs' records (Sec. VIII, Eqs.
// weighted-averages, modified-weights2: k_weighted, one thread, runs in order).
//
// The analysis is three launches on the context's stream:
//   k_ana_blocks    one CUDA block per analysis block: exact int64 sums of E, E^2, |M|, M^2
//                   over the block's slot range [floor(b R / n), floor((b + 1) R / n));
//   k_ana_families  family sizes (runs of equal ids in slot order) into a size histogram;
//   k_ana_final     one block: the binary64 formulas over the n blocks in block order (one
//                   thread), and -sum_s c_s (s / R) ln(s / R) over family sizes s.
#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {

namespace {

constexpr int kAnaThreads = 256;
constexpr int kAnaFinalThreads = 1024;

template <typename T, int THREADS>
__device__ __forceinline__ T ana_block_sum(T v)
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

__global__ void __launch_bounds__(kAnaThreads) k_ana_blocks(const DevState *st, const int *level, const int *mag,
                                                            int N, int n, long long *blk)
{
    const long long R = st->R_cur;
    const int b = blockIdx.x;
    const long long lo = ((long long)b * R) / n, hi = ((long long)(b + 1) * R) / n;
    long long sE = 0, sE2 = 0, sA = 0, sA2 = 0;
    for (long long j = lo + threadIdx.x; j < hi; j += kAnaThreads) {
        const long long E = 4LL * level[j] - 2LL * N;
        const long long m = mag[j];
        const long long a = m < 0 ? -m : m;
        sE += E;
        sE2 += E * E;
        sA += a;
        sA2 += a * a;
    }
    sE = ana_block_sum<long long, kAnaThreads>(sE);
    sE2 = ana_block_sum<long long, kAnaThreads>(sE2);
    sA = ana_block_sum<long long, kAnaThreads>(sA);
    sA2 = ana_block_sum<long long, kAnaThreads>(sA2);
    if (threadIdx.x == 0) {
        blk[4 * b + 0] = sE;
        blk[4 * b + 1] = sE2;
        blk[4 * b + 2] = sA;
        blk[4 * b + 3] = sA2;
    }
}

// sizes[0] = largest family size, sizes[s] = number of families of size s (s >= 1); zeroed
// by the caller before the launch.
__global__ void __launch_bounds__(kAnaThreads) k_ana_families(const DevState *st, const int *fam, int *sizes)
{
    const long long R = st->R_cur;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < R;
         j += (long long)gridDim.x * blockDim.x) {
        const int f = fam[j];
        if (j > 0 && fam[j - 1] == f) continue;
        // a family starts at j: find its end by doubling steps, then halving
        long long in = j, step = 1;
        while (in + step < R && fam[in + step] == f) {
            in += step;
            step <<= 1;
        }
        long long out = in + step < R ? in + step : R;  // first index known outside (or R)
        while (out - in > 1) {
            const long long mid = in + (out - in) / 2;
            if (fam[mid] == f) in = mid;
            else out = mid;
        }
        const int size = (int)(out - j);
        atomicAdd(&sizes[size], 1);
        atomicMax(&sizes[0], size);
    }
}

__global__ void __launch_bounds__(kAnaFinalThreads) k_ana_final(const DevState *st, const long long *blk, int n,
                                                                 int N, double beta, const int *sizes,
                                                                 pa_analysis *out)
{
    const long long R = st->R_cur;
    const double Rd = (double)R;

    // family entropy from the size histogram, in a fixed order (thread strides, then a
    // fixed tree over the block)
    const int smax = sizes[0];
    double part = 0.0;
    long long fam = 0;
    for (int s = 1 + (int)threadIdx.x; s <= smax; s += kAnaFinalThreads) {
        const int c = sizes[s];
        if (c) {
            const double nk = (double)s / Rd;
            part = __dadd_rn(part, __dmul_rn((double)c, __dmul_rn(nk, log(nk))));
            fam += c;
        }
    }
    __shared__ double sh_part[kAnaFinalThreads];
    __shared__ long long sh_fam[kAnaFinalThreads];
    sh_part[threadIdx.x] = part;
    sh_fam[threadIdx.x] = fam;
    __syncthreads();
    for (int w = kAnaFinalThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh_part[threadIdx.x] = __dadd_rn(sh_part[threadIdx.x], sh_part[threadIdx.x + w]);
            sh_fam[threadIdx.x] += sh_fam[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;

    const double Nd = (double)N, nd = (double)n;
    long long tE = 0, tE2 = 0, tA = 0, tA2 = 0;
    for (int b = 0; b < n; ++b) {
        tE += blk[4 * b + 0];
        tE2 += blk[4 * b + 1];
        tA += blk[4 * b + 2];
        tA2 += blk[4 * b + 3];
    }
    const double meanE = (double)tE / Rd, meanE2 = (double)tE2 / Rd;
    const double meanA = (double)tA / Rd;
    const double varE = (R > 1) ? __ddiv_rn(__dsub_rn((double)tE2, __dmul_rn(Rd, __dmul_rn(meanE, meanE))), Rd - 1.0)
                                : 0.0;
    const double varA = (R > 1) ? __ddiv_rn(__dsub_rn((double)tA2, __dmul_rn(Rd, __dmul_rn(meanA, meanA))), Rd - 1.0)
                                : 0.0;
    auto cnt = [&](int b) { return ((long long)(b + 1) * R) / n - ((long long)b * R) / n; };

    // blocked estimator
    double mBE = 0.0, mBA = 0.0;
    for (int b = 0; b < n; ++b) {
        mBE = __dadd_rn(mBE, (double)blk[4 * b + 0] / (double)cnt(b));
        mBA = __dadd_rn(mBA, (double)blk[4 * b + 2] / (double)cnt(b));
    }
    mBE /= nd;
    mBA /= nd;
    double vBE = 0.0, vBA = 0.0;
    for (int b = 0; b < n; ++b) {
        const double dE = __dsub_rn((double)blk[4 * b + 0] / (double)cnt(b), mBE);
        const double dA = __dsub_rn((double)blk[4 * b + 2] / (double)cnt(b), mBA);
        vBE = __dadd_rn(vBE, __dmul_rn(dE, dE));
        vBA = __dadd_rn(vBA, __dmul_rn(dA, dA));
    }
    vBE /= __dmul_rn(nd, nd - 1.0);
    vBA /= __dmul_rn(nd, nd - 1.0);

    // jackknife: leave-one-block-out means, and C from them
    auto jack = [&](int b, double &jE, double &jA, double &jC) {
        const double rest = (double)(R - cnt(b));
        jE = (double)(tE - blk[4 * b + 0]) / rest;
        const double jE2 = (double)(tE2 - blk[4 * b + 1]) / rest;
        jA = (double)(tA - blk[4 * b + 2]) / rest;
        jC = __dmul_rn(beta, beta) * __dsub_rn(jE2, __dmul_rn(jE, jE)) / Nd;
    };
    double mJE = 0.0, mJA = 0.0, mJC = 0.0;
    for (int b = 0; b < n; ++b) {
        double jE, jA, jC;
        jack(b, jE, jA, jC);
        mJE = __dadd_rn(mJE, jE);
        mJA = __dadd_rn(mJA, jA);
        mJC = __dadd_rn(mJC, jC);
    }
    mJE /= nd;
    mJA /= nd;
    mJC /= nd;
    double vJE = 0.0, vJA = 0.0, vJC = 0.0;
    for (int b = 0; b < n; ++b) {
        double jE, jA, jC;
        jack(b, jE, jA, jC);
        vJE = __dadd_rn(vJE, __dmul_rn(jE - mJE, jE - mJE));
        vJA = __dadd_rn(vJA, __dmul_rn(jA - mJA, jA - mJA));
        vJC = __dadd_rn(vJC, __dmul_rn(jC - mJC, jC - mJC));
    }
    const double fj = (nd - 1.0) / nd;
    vJE = __dmul_rn(vJE, fj);
    vJA = __dmul_rn(vJA, fj);
    vJC = __dmul_rn(vJC, fj);

    const double Sf = -sh_part[0];
    pa_analysis o;
    o.R = R;
    o.n_blocks = n;
    o.families = sh_fam[0];
    o.beta = beta;
    o.mean_E = meanE;
    o.var_E = varE;
    o.var_mean_E_jack = vJE;
    o.var_mean_E_blocked = vBE;
    o.R_eff_E = varE / vJE;
    o.mean_absM = meanA;
    o.var_absM = varA;
    o.var_mean_absM_jack = vJA;
    o.var_mean_absM_blocked = vBA;
    o.R_eff_M = varA / vJA;
    o.C = __dmul_rn(beta, beta) * __dsub_rn(meanE2, __dmul_rn(meanE, meanE)) / Nd;
    o.var_C_jack = vJC;
    o.S_f = Sf;
    o.rho_s = Rd / exp(Sf);
    *out = o;
}

__global__ void k_weighted(const pa_obs *rec, int M, int mode, pa_weighted *out)
{
    if (threadIdx.x != 0) return;
    pa_weighted o{};
    o.M = M;
    o.mode = mode;
    o.step = rec[0].step;
    o.beta = rec[0].beta;
    int status = 0;
    for (int m = 0; m < M; ++m) {
        if (rec[m].step != o.step || rec[m].beta != o.beta) status = PA_ERR_INVALID_ARG;
        if (!status && rec[m].status) status = rec[m].status;
    }
    o.status = status;
    auto lw = [&](int m) {
        return __dadd_rn(__dadd_rn(log((double)rec[m].R), rec[m].minus_betaF), mode == 1 ? rec[m].sum_lnRratio : 0.0);
    };
    auto lz = [&](int m) { return __dadd_rn(log((double)rec[m].R_target), rec[m].minus_betaF); };
    double mx = -INFINITY, mz = -INFINITY, sR = 0.0;
    for (int m = 0; m < M; ++m) {
        mx = fmax(mx, lw(m));
        mz = fmax(mz, lz(m));
        sR = __dadd_rn(sR, (double)rec[m].R_target);
    }
    double s = 0.0, sz = 0.0;
    for (int m = 0; m < M; ++m) {
        s = __dadd_rn(s, exp(__dsub_rn(lw(m), mx)));
        sz = __dadd_rn(sz, exp(__dsub_rn(lz(m), mz)));
    }
    double w2 = 0.0, wmax = 0.0, meanF = 0.0;
    double acc[5] = {0, 0, 0, 0, 0}, pl[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < M; ++m) {
        const double om = __ddiv_rn(exp(__dsub_rn(lw(m), mx)), s);
        w2 = __dadd_rn(w2, __dmul_rn(om, om));
        wmax = fmax(wmax, om);
        const double v[5] = {rec[m].e, rec[m].C, rec[m].m, rec[m].m2, rec[m].chi};
        for (int q = 0; q < 5; ++q) {
            acc[q] = __dadd_rn(acc[q], __dmul_rn(om, v[q]));
            pl[q] = __dadd_rn(pl[q], v[q]);
        }
        meanF = __dadd_rn(meanF, rec[m].minus_betaF);
    }
    meanF = __ddiv_rn(meanF, (double)M);
    double vF = 0.0;
    for (int m = 0; m < M; ++m) {
        const double d = __dsub_rn(rec[m].minus_betaF, meanF);
        vF = __dadd_rn(vF, __dmul_rn(d, d));
    }
    o.var_minus_betaF = M > 1 ? __ddiv_rn(vF, (double)(M - 1)) : 0.0;
    o.M_eff = __ddiv_rn(1.0, w2);
    o.max_weight = wmax;
    o.minus_betaF_combined = __dsub_rn(__dadd_rn(mz, log(sz)), log(sR));
    o.e = acc[0]; o.C = acc[1]; o.m = acc[2]; o.m2 = acc[3]; o.chi = acc[4];
    o.e_plain = __ddiv_rn(pl[0], (double)M);
    o.C_plain = __ddiv_rn(pl[1], (double)M);
    o.m_plain = __ddiv_rn(pl[2], (double)M);
    o.m2_plain = __ddiv_rn(pl[3], (double)M);
    o.chi_plain = __ddiv_rn(pl[4], (double)M);
    *out = o;
}

}  // namespace

cudaError_t launch_weighted(const pa_obs *rec, int M, int mode, pa_weighted *out, cudaStream_t s)
{
    k_weighted<<<1, 32, 0, s>>>(rec, M, mode, out);
    return cudaGetLastError();
}

cudaError_t launch_analysis(const DevState *st, const int *level, const int *mag, const int *fam, int N,
                            double beta, int n, long long capacity, long long *blk, int *sizes, pa_analysis *out,
                            cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(sizes, 0, (size_t)(capacity + 1) * sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_ana_blocks<<<n, kAnaThreads, 0, s>>>(st, level, mag, N, n, blk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ana_families<<<kFamBlocks, kAnaThreads, 0, s>>>(st, fam, sizes);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ana_final<<<1, kAnaFinalThreads, 0, s>>>(st, blk, n, N, beta, sizes, out);
    return cudaGetLastError();
}

}  // namespace pa
