/* Population analysis of population annealing (arXiv:2102.06611): the quantities the paper
 * uses to assess a run from its final population.  TEST INFRASTRUCTURE (oracle): plain
 * single-threaded C written from the paper's definitions, one step after another; it
 * shares no code with the CUDA path.
 *
 *   Blocked errors (Sec. IV, Eqs. blocks, blocked_variance): the R replicas are taken in
 *   slot order, which is tree order (children of one parent sit next to each other), cut
 *   into n contiguous blocks; the block means O^B_b give the variance of the mean
 *   sigma^2_B = 1/(n (n-1)) sum_b (O^B_b - mean_b O^B)^2.
 *   Jackknife (Eqs. jackknife-blocks, jackknife-variance): O^J_b = mean of all replicas
 *   outside block b, sigma^2_J = (n-1)/n sum_b (O^J_b - mean_b O^J)^2; also for the
 *   specific heat C = beta^2 (<E^2> - <E>^2) / N, a non-linear function of two means.
 *   Effective population size (Eq. neff): R_eff(O) = sigma^2(O) / sigma^2_J(mean O), with
 *   sigma^2(O) the unbiased variance of the unblocked series.
 *   Family entropy (Sec. V, Eq. rhos): S_f = -sum_k n_k ln n_k over families k with
 *   n_k = size_k / R, and rho_s = R / exp(S_f).
 *
 * Readings where the paper is silent: when n does not divide R the blocks are slot ranges
 * [floor(b R / n), floor((b+1) R / n)), whose sizes differ by at most one, and O^J_b is the
 * mean over the R - B_b replicas outside block b (equal to the paper's B/(R-B) sum_{c != b}
 * O^B_c when all blocks have B replicas).  The observables are the energy E and |M|.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* out[0] n, [1] mean E, [2] sigma^2(E), [3] sigma^2_J(mean E), [4] sigma^2_B(mean E),
 * [5] R_eff(E), [6] mean |M|, [7] sigma^2(|M|), [8] sigma^2_J(mean |M|),
 * [9] sigma^2_B(mean |M|), [10] R_eff(|M|), [11] C, [12] sigma^2_J(C), [13] S_f,
 * [14] rho_s, [15] families.  Returns 0, or 1 if n < 2 or n > R. */
int orc_analysis(int N, double beta, int64_t R, const int32_t *E, const int32_t *M, const int32_t *fam,
                 int n, double *out)
{
    if (n < 2 || (int64_t)n > R) return 1;
    const double Rd = (double)R, Nd = (double)N, nd = (double)n;

    /* exact integer sums per block and in total */
    int64_t *sE = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *sE2 = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *sA = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t tE = 0, tE2 = 0, tA = 0, tA2 = 0;
    for (int b = 0; b < n; ++b) {
        const int64_t lo = ((int64_t)b * R) / n, hi = ((int64_t)(b + 1) * R) / n;
        for (int64_t j = lo; j < hi; ++j) {
            const int64_t e = E[j], a = M[j] < 0 ? -(int64_t)M[j] : (int64_t)M[j];
            sE[b] += e;
            sE2[b] += e * e;
            sA[b] += a;
        }
        cnt[b] = hi - lo;
        tE += sE[b];
        tE2 += sE2[b];
        tA += sA[b];
    }
    for (int64_t j = 0; j < R; ++j) {
        const int64_t a = M[j] < 0 ? -(int64_t)M[j] : (int64_t)M[j];
        tA2 += a * a;
    }

    const double meanE = (double)tE / Rd, meanE2 = (double)tE2 / Rd;
    const double meanA = (double)tA / Rd;
    /* unbiased variances of the unblocked series: (sum x^2 - R mean^2) / (R - 1) */
    const double varE = (R > 1) ? ((double)tE2 - Rd * (meanE * meanE)) / (Rd - 1.0) : 0.0;
    const double varA = (R > 1) ? ((double)tA2 - Rd * (meanA * meanA)) / (Rd - 1.0) : 0.0;

    /* blocked: means of the block means, then the naive variance of the mean */
    double mBE = 0.0, mBA = 0.0;
    for (int b = 0; b < n; ++b) {
        mBE += (double)sE[b] / (double)cnt[b];
        mBA += (double)sA[b] / (double)cnt[b];
    }
    mBE /= nd;
    mBA /= nd;
    double vBE = 0.0, vBA = 0.0;
    for (int b = 0; b < n; ++b) {
        const double dE = (double)sE[b] / (double)cnt[b] - mBE;
        const double dA = (double)sA[b] / (double)cnt[b] - mBA;
        vBE += dE * dE;
        vBA += dA * dA;
    }
    vBE /= nd * (nd - 1.0);
    vBA /= nd * (nd - 1.0);

    /* jackknife: leave-one-block-out means and the specific heat built from them */
    double mJE = 0.0, mJA = 0.0, mJC = 0.0;
    for (int b = 0; b < n; ++b) {
        const double rest = (double)(R - cnt[b]);
        const double jE = (double)(tE - sE[b]) / rest;
        const double jE2 = (double)(tE2 - sE2[b]) / rest;
        const double jA = (double)(tA - sA[b]) / rest;
        const double jC = ((beta * beta) * (jE2 - jE * jE)) / Nd;
        mJE += jE;
        mJA += jA;
        mJC += jC;
    }
    mJE /= nd;
    mJA /= nd;
    mJC /= nd;
    double vJE = 0.0, vJA = 0.0, vJC = 0.0;
    for (int b = 0; b < n; ++b) {
        const double rest = (double)(R - cnt[b]);
        const double jE = (double)(tE - sE[b]) / rest;
        const double jE2 = (double)(tE2 - sE2[b]) / rest;
        const double jA = (double)(tA - sA[b]) / rest;
        const double jC = ((beta * beta) * (jE2 - jE * jE)) / Nd;
        vJE += (jE - mJE) * (jE - mJE);
        vJA += (jA - mJA) * (jA - mJA);
        vJC += (jC - mJC) * (jC - mJC);
    }
    const double fj = (nd - 1.0) / nd;
    vJE *= fj;
    vJA *= fj;
    vJC *= fj;

    /* families: runs of equal ids in slot order; S_f = -sum_k (size_k / R) ln(size_k / R),
       accumulated in long double: up to R terms, many of them equal, whose binary64
       rounding errors would add up coherently */
    long double acc = 0.0L;
    int64_t f = 0, run = 0;
    for (int64_t j = 0; j <= R; ++j) {
        if (j == R || (j > 0 && fam[j] != fam[j - 1])) {
            const long double nk = (long double)run / (long double)R;
            acc -= nk * logl(nk);
            ++f;
            run = 0;
            if (j == R) break;
        }
        ++run;
    }
    const double Sf = (double)acc;

    out[0] = nd;
    out[1] = meanE;
    out[2] = varE;
    out[3] = vJE;
    out[4] = vBE;
    out[5] = varE / vJE;
    out[6] = meanA;
    out[7] = varA;
    out[8] = vJA;
    out[9] = vBA;
    out[10] = varA / vJA;
    out[11] = ((beta * beta) * (meanE2 - meanE * meanE)) / Nd;
    out[12] = vJC;
    out[13] = Sf;
    out[14] = Rd / exp(Sf);
    out[15] = (double)f;
    free(sE);
    free(sE2);
    free(sA);
    free(cnt);
    return 0;
}
