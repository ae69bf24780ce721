/*
 * exact_ising.c -- exact finite-lattice results for the 2D Ising ferromagnet (J = 1,
 * L x L, periodic boundaries), used to pin the population-annealing oracle.
 *
 * TEST INFRASTRUCTURE (part of the oracle): only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load it.
 *
 * The paper compares its simulations with exact finite-size results (Sec. III, the
 * citations of Kaufman 1949, Ferdinand & Fisher 1969 and Beale 1996) but prints none of
 * the formulas.  Three independent exact methods are provided so that each pins the
 * others:
 *   1. brute-force enumeration of all 2^N states (L = 4): density of states per energy
 *      level and the magnetisation sums per level;
 *   2. the row-to-row transfer matrix, Z = Tr T^L, in long double (L <= 8);
 *   3. Kaufman's closed form for the periodic L x L lattice, as written by Ferdinand and
 *      Fisher (Phys. Rev. 185, 832 (1969), Eqs. 2.1-2.4):
 *        Z = 1/2 (2 sinh 2K)^{N/2} (Z1 + Z2 + Z3 + Z4),
 *        Z1 = prod_{r=0}^{L-1} 2 cosh(L g_{2r+1} / 2),  Z2 = same with sinh,
 *        Z3 = prod_{r=0}^{L-1} 2 cosh(L g_{2r} / 2),    Z4 = same with sinh,
 *        cosh g_l = cosh 2K coth 2K - cos(pi l / L)   (l >= 1),
 *        g_0 = 2K + ln tanh K                         (with its sign),
 *      evaluated in long double with the four products combined in log space.
 * Energy and specific heat follow from ln Z by Richardson-extrapolated central
 * differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* 1. Enumeration: g[k] = number of states at level k (E = 4k - 2N), sabsm[k] = sum of
   |M| over those states, sm2[k] = sum of M^2, for 0 <= k <= N.  Returns 0, or 1 if L
   is too large to enumerate (N > 24). */
int orc_bruteforce(int L, int64_t *g, int64_t *sabsm, int64_t *sm2)
{
    int N = L * L;
    if (N > 24) return 1;
    memset(g, 0, sizeof(int64_t) * (size_t)(N + 1));
    memset(sabsm, 0, sizeof(int64_t) * (size_t)(N + 1));
    memset(sm2, 0, sizeof(int64_t) * (size_t)(N + 1));
    for (uint64_t state = 0; state < (1ull << N); ++state) {
        int E = 0, M = 0;
        for (int r = 0; r < L; ++r)
            for (int c = 0; c < L; ++c) {
                int s = ((state >> (r * L + c)) & 1u) ? 1 : -1;
                int right = ((state >> (r * L + (c + 1) % L)) & 1u) ? 1 : -1;
                int down = ((state >> (((r + 1) % L) * L + c)) & 1u) ? 1 : -1;
                E -= s * right + s * down;
                M += s;
            }
        int k = (E + 2 * N) / 4;
        g[k] += 1;
        sabsm[k] += (M < 0 ? -M : M);
        sm2[k] += (int64_t)M * M;
    }
    return 0;
}

/* 2. Transfer matrix: ln Z(beta) = ln Tr T^L with the symmetric row transfer matrix
   T(a, b) = exp(beta [H(a)/2 + H(b)/2 + V(a, b)]), H(a) = sum_c a_c a_{c+1} (periodic
   along the row), V(a, b) = sum_c a_c b_c.  Returns NaN if L > 10 or L < 2. */
double orc_transfer_lnZ(int L, double beta)
{
    if (L < 2 || L > 10) return NAN;
    int S = 1 << L;
    long double *T = (long double *)malloc(sizeof(long double) * (size_t)S * S);
    long double *P = (long double *)malloc(sizeof(long double) * (size_t)S * S);
    long double *Q = (long double *)malloc(sizeof(long double) * (size_t)S * S);
    int *H = (int *)malloc(sizeof(int) * (size_t)S);
    for (int a = 0; a < S; ++a) {
        int h = 0;
        for (int c = 0; c < L; ++c) {
            int sa = ((a >> c) & 1) ? 1 : -1;
            int sb = ((a >> ((c + 1) % L)) & 1) ? 1 : -1;
            h += sa * sb;
        }
        H[a] = h;
    }
    /* Scale every entry by exp(-beta * 2L) (the largest possible exponent is 2L beta),
       which multiplies Tr T^L by exp(-2 L^2 beta) and is undone at the end. */
    long double b = (long double)beta;
    for (int a = 0; a < S; ++a)
        for (int c = 0; c < S; ++c) {
            int v = 0;
            for (int i = 0; i < L; ++i) {
                int sa = ((a >> i) & 1) ? 1 : -1;
                int sc = ((c >> i) & 1) ? 1 : -1;
                v += sa * sc;
            }
            long double x = 0.5L * (long double)H[a] + 0.5L * (long double)H[c] + (long double)v;
            T[(size_t)a * S + c] = expl(b * (x - 2.0L * (long double)L));
        }
    memcpy(P, T, sizeof(long double) * (size_t)S * S);
    for (int step = 1; step < L; ++step) {
        for (int a = 0; a < S; ++a)
            for (int c = 0; c < S; ++c) {
                long double acc = 0.0L;
                for (int k = 0; k < S; ++k) acc += P[(size_t)a * S + k] * T[(size_t)k * S + c];
                Q[(size_t)a * S + c] = acc;
            }
        long double *t = P; P = Q; Q = t;
    }
    long double tr = 0.0L;
    for (int a = 0; a < S; ++a) tr += P[(size_t)a * S + a];
    double out = (double)(logl(tr) + 2.0L * (long double)L * (long double)L * b);
    free(T); free(P); free(Q); free(H);
    return out;
}

/* log of |2 cosh x| and of |2 sinh x| for real x, without overflow. */
static long double ln2cosh(long double x)
{
    long double a = fabsl(x);
    return a + log1pl(expl(-2.0L * a));
}
static long double ln2sinh_abs(long double x)
{
    long double a = fabsl(x);
    return a + log1pl(-expl(-2.0L * a));
}

/* 3. Kaufman / Ferdinand-Fisher ln Z for the periodic L x L lattice in long double. */
long double orc_kaufman_lnZ_l(int L, long double K)
{
    int N = L * L;
    long double c2 = coshl(2.0L * K), s2 = sinhl(2.0L * K);
    long double base = c2 * c2 / s2; /* cosh 2K coth 2K */
    long double pi = acosl(-1.0L);
    long double lnZ1 = 0.0L, lnZ2 = 0.0L, lnZ3 = 0.0L, lnZ4 = 0.0L;
    int sign4 = 1;
    for (int r = 0; r < L; ++r) {
        int lo = 2 * r + 1, le = 2 * r;
        long double go = acoshl(base - cosl(pi * (long double)lo / (long double)L));
        long double ge;
        if (le == 0) ge = 2.0L * K + logl(tanhl(K));
        else ge = acoshl(base - cosl(pi * (long double)le / (long double)L));
        long double xo = 0.5L * (long double)L * go, xe = 0.5L * (long double)L * ge;
        lnZ1 += ln2cosh(xo);
        lnZ2 += ln2sinh_abs(xo);
        lnZ3 += ln2cosh(xe);
        if (xe == 0.0L) sign4 = 0;
        else {
            lnZ4 += ln2sinh_abs(xe);
            if (xe < 0.0L) sign4 = -sign4;
        }
    }
    long double mx = lnZ1;
    if (lnZ2 > mx) mx = lnZ2;
    if (lnZ3 > mx) mx = lnZ3;
    if (sign4 != 0 && lnZ4 > mx) mx = lnZ4;
    long double sum = expl(lnZ1 - mx) + expl(lnZ2 - mx) + expl(lnZ3 - mx);
    if (sign4 != 0) sum += (long double)sign4 * expl(lnZ4 - mx);
    return -logl(2.0L) + 0.5L * (long double)N * logl(2.0L * s2) + mx + logl(sum);
}

double orc_kaufman_lnZ(int L, double beta)
{
    return (double)orc_kaufman_lnZ_l(L, (long double)beta);
}

/* Energy <E> = -d lnZ / d beta and specific heat per spin C = beta^2 / N d^2 lnZ /
   d beta^2 from Richardson-extrapolated central differences of the closed form.
   out[0] = <E>, out[1] = C, out[2] = ln Z. */
void orc_kaufman_thermo(int L, double beta, double h, double *out)
{
    long double b = (long double)beta, hh = (long double)h;
    long double f0 = orc_kaufman_lnZ_l(L, b);
    long double fp1 = orc_kaufman_lnZ_l(L, b + hh), fm1 = orc_kaufman_lnZ_l(L, b - hh);
    long double fp2 = orc_kaufman_lnZ_l(L, b + 0.5L * hh), fm2 = orc_kaufman_lnZ_l(L, b - 0.5L * hh);
    long double d1h = (fp1 - fm1) / (2.0L * hh);
    long double d1h2 = (fp2 - fm2) / hh;
    long double d2h = (fp1 - 2.0L * f0 + fm1) / (hh * hh);
    long double d2h2 = (fp2 - 2.0L * f0 + fm2) / (0.25L * hh * hh);
    long double d1 = (4.0L * d1h2 - d1h) / 3.0L;
    long double d2 = (4.0L * d2h2 - d2h) / 3.0L;
    int N = L * L;
    out[0] = (double)(-d1);
    out[1] = (double)(b * b * d2 / (long double)N);
    out[2] = (double)f0;
}
