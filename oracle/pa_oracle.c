/*
 * pa_oracle.c -- plain, slow, single-threaded CPU population annealing (PA) for the
 * 2D Ising ferromagnet (J = 1, L x L, periodic), written from Weigel, Barash, Shchur,
 * Janke, "Understanding population annealing Monte Carlo simulations" (arXiv:2102.06611).
 *
 * TEST INFRASTRUCTURE.  This file is the oracle the CUDA path is checked against.  Only
 * tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may load
 * it.  It shares no code, header or constant generator with the CUDA library; where a
 * definition must agree bit for bit (Philox4x32-10, the deterministic exp, the random-
 * number keying, the decision rules) it is written here independently from the same
 * published definition.
 *
 * Spins are one int8 per site (+1 / -1), replica-major, row-major: s[j*N + r*L + c].
 * Everything is done site by site in the paper's order; nothing is blocked or fused.
 *
 * Paper passages followed:
 *   Sec. II steps 1-5 (population annealing loop), Eq. (Q) normalisation Q_i,
 *   Eq. (taus) rescaled copy means, Eq. (resampling-factors) nearest-integer copies,
 *   Poisson resampling (Sec. II, Machta's variant), Eq. (hamiltonian), Sec. III
 *   observables e, C_V, m, chi, Sec. V families and Eq. (rhot), Sec. VII
 *   Eq. (free-emergy-estimator) with ln Z_0 = L^d ln 2.
 *
 * Parity of the pieces not printed in the paper is pinned by tests/test_oracle_*.py:
 * Philox by the published known-answer vectors, orc_exp against libm and a
 * 60-digit reference, the sweep by brute-force Boltzmann distributions at L = 4, the
 * Q_i / free-energy path by the exact finite-lattice partition function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11).  Ten rounds; each round multiplies counter words 0 and 2 by the
 * two round multipliers (full 64-bit products), and the key is bumped by the two Weyl
 * constants between rounds.
 * ---------------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ x1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ x3 ^ k1;
        uint32_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random-number streams: the tag sits in the top 4 bits of counter word 2. */
enum { STREAM_INIT = 0, STREAM_SWEEP = 1, STREAM_RESAMPLE = 2, STREAM_POISSON = 3 };

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                            uint32_t c3, int lane)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[lane];
}

/* ------------------------------------------------------------------------------------
 * Deterministic exp (Cody & Waite argument reduction, then the Taylor series of e^r
 * to degree 13 in Horner form).  x = k ln2 + r with k = rint(x / ln2), |r| <= ln2/2;
 * ln2 is split as LN2_HI (32 significant bits, so k * LN2_HI is exact) plus LN2_LO.
 * e^r = sum_{n<=13} r^n / n!; the truncation error r^14/14! < 5e-18 is below half an
 * ulp.  Each multiply and add is a separate IEEE binary64 operation (the file is built
 * with -ffp-contract=off), so the result is a fixed function of x.
 * ---------------------------------------------------------------------------------- */
#define ORC_LN2_HI 0x1.62e42feep-1
#define ORC_LN2_LO 0x1.a39ef35793c76p-33
#define ORC_INV_LN2 0x1.71547652b82fep+0

double orc_exp(double x)
{
    if (x != x) return x;
    if (x > 709.5) return HUGE_VAL;
    if (x < -745.5) return 0.0;
    double k = rint(x * ORC_INV_LN2);
    double r = (x - k * ORC_LN2_HI) - k * ORC_LN2_LO;
    /* 1/n! for n = 13 .. 1; n! is an exact double for n <= 18, so each coefficient is
       the correctly rounded quotient. */
    double p = 1.0 / 6227020800.0;          /* 1/13! */
    p = p * r + 1.0 / 479001600.0;          /* 1/12! */
    p = p * r + 1.0 / 39916800.0;           /* 1/11! */
    p = p * r + 1.0 / 3628800.0;            /* 1/10! */
    p = p * r + 1.0 / 362880.0;             /* 1/9!  */
    p = p * r + 1.0 / 40320.0;              /* 1/8!  */
    p = p * r + 1.0 / 5040.0;               /* 1/7!  */
    p = p * r + 1.0 / 720.0;                /* 1/6!  */
    p = p * r + 1.0 / 120.0;                /* 1/5!  */
    p = p * r + 1.0 / 24.0;                 /* 1/4!  */
    p = p * r + 1.0 / 6.0;                  /* 1/3!  */
    p = p * r + 0.5;                        /* 1/2!  */
    p = p * r + 1.0;                        /* 1/1!  */
    p = p * r + 1.0;                        /* 1/0!  */
    return ldexp(p, (int)k);
}

/* Metropolis threshold floor(exp(-y) * 2^32) for y >= 0; 2^32 means "always". */
uint64_t orc_metropolis_threshold(double y)
{
    double p = orc_exp(-y);
    return (uint64_t)floor(p * 4294967296.0);
}

/* Heatbath (Sec. IV; for Ising spins the same as Glauber): a site with a aligned neighbours
   flips with probability p_a = 1 / (1 + exp(beta dE)), dE = 4a - 8, so p_a + p_{4-a} = 1 and
   p_2 = 1/2.  Reading: flip iff x < T_a with the 32-bit uniform x of the site and
     T_3 = floor(p_3 2^32), T_4 = floor(p_4 2^32)          (p_3, p_4 <= 1/2),
     T_1 = 2^32 - T_3,      T_0 = 2^32 - T_4,    T_2 = 2^31,
   i.e. every p_a to 2^-32 and exactly complementary in pairs.  orc_heatbath_threshold(y)
   is floor(2^32 / (1 + exp(y))) for y = 4 beta (T_3) or 8 beta (T_4). */
uint64_t orc_heatbath_threshold(double y)
{
    double p = 1.0 / (1.0 + orc_exp(y));
    return (uint64_t)floor(p * 4294967296.0);
}

/* ------------------------------------------------------------------------------------
 * Lattice helpers.  E = -sum over the 2N nearest-neighbour bonds of s_i s_j
 * (Eq. hamiltonian with J = 1), M = sum of spins.  The energy level is
 * k = (E + 2N) / 4 in [0, N] (E = 2 n_anti - 2N and n_anti is even on the torus).
 * ---------------------------------------------------------------------------------- */
static inline int site(int L, int r, int c)
{
    r = (r + L) % L;
    c = (c + L) % L;
    return r * L + c;
}

void orc_energy_mag(int L, const int8_t *s, int32_t *E_out, int32_t *M_out)
{
    int E = 0, M = 0;
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c) {
            int si = s[site(L, r, c)];
            E -= si * s[site(L, r, c + 1)];
            E -= si * s[site(L, r + 1, c)];
            M += si;
        }
    *E_out = E;
    *M_out = M;
}

/* FNV-1a 64 of the canonical packed bytes of one replica: for each row, ceil(L/32)
   little-endian uint32 words, bit b of word w set iff the spin at column 32w + b is +1. */
uint64_t orc_hash(int L, const int8_t *s)
{
    uint64_t h = 0xcbf29ce484222325ull;
    int words = (L + 31) / 32;
    for (int r = 0; r < L; ++r)
        for (int w = 0; w < words; ++w) {
            uint32_t v = 0;
            for (int b = 0; b < 32; ++b) {
                int c = 32 * w + b;
                if (c < L && s[r * L + c] > 0) v |= (1u << b);
            }
            for (int byte = 0; byte < 4; ++byte) {
                h ^= (uint64_t)((v >> (8 * byte)) & 0xffu);
                h *= 0x100000001b3ull;
            }
        }
    return h;
}

/* Canonical packed form (same bytes as hashed) <-> int8 spins. */
void orc_pack(int L, const int8_t *s, uint32_t *out)
{
    int words = (L + 31) / 32;
    for (int r = 0; r < L; ++r)
        for (int w = 0; w < words; ++w) {
            uint32_t v = 0;
            for (int b = 0; b < 32; ++b) {
                int c = 32 * w + b;
                if (c < L && s[r * L + c] > 0) v |= (1u << b);
            }
            out[r * words + w] = v;
        }
}

void orc_unpack(int L, const uint32_t *in, int8_t *s)
{
    int words = (L + 31) / 32;
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c)
            s[r * L + c] = ((in[r * words + c / 32] >> (c % 32)) & 1u) ? 1 : -1;
}

/* ------------------------------------------------------------------------------------
 * Step 1 (Sec. II): simple sampling at beta_0 = 0.  Site n = r L + c of replica j takes
 * bit (n mod 32) of the 32-bit word number n / 32 of the INIT stream: word w is lane
 * (w mod 4) of Philox(ctr = (w / 4, j, INIT << 28, 0)); a set bit is s = +1.
 * ---------------------------------------------------------------------------------- */
void orc_init_replica(int L, uint64_t seed, uint32_t j, int8_t *s)
{
    int N = L * L;
    for (int n = 0; n < N; ++n) {
        uint32_t w = (uint32_t)n >> 5;
        uint32_t x = philox_word(seed, w >> 2, j, (uint32_t)STREAM_INIT << 28, 0, (int)(w & 3));
        s[n] = ((x >> (n & 31)) & 1u) ? 1 : -1;
    }
}

/* ------------------------------------------------------------------------------------
 * Step 3 (Sec. II): theta rounds of single-spin Metropolis at inverse temperature beta,
 * in checkerboard order (the paper's GPU variant): within sweep t, first every site with
 * (r + c) even (colour 0), then every site with (r + c) odd (colour 1).  Sites of one
 * colour do not interact, so visiting them one after another is the same as updating
 * them together.  Acceptance is min(1, exp(-beta dE)) with dE = 4a - 8, a = number of
 * aligned neighbours: a <= 2 always flips; a = 3 flips iff x < floor(e^{-4 beta} 2^32);
 * a = 4 flips iff x < floor(e^{-8 beta} 2^32), x a uniform 32-bit integer.
 *
 * The uniform x of site (r, c) of colour q in sweep t of step i, replica slot j, is built
 * from two independent parts (every bit is an independent uniform bit, so x is uniform on
 * [0, 2^32)).  Let p = c / 2 (index of the site among the L/2 colour-q sites of row r),
 * H' = the smallest power of two >= L/2, n = r H' + p (the colour-q sites numbered row
 * after row, each row padded to H'), chunk = n / 32, b = n mod 32, tag = (2t + q).  For
 * L >= 64 a chunk is 32 sites of one row; for smaller L it spans 32 / H' rows:
 *   top 8 bits:   bit (31 - k) of x, k = 0..7, is bit b of word (k mod 4) of
 *                 Philox(ctr = (2 chunk + k / 4, j, (SWEEP << 28) | tag, i));
 *   low 24 bits:  the low 24 bits of word 0 of
 *                 Philox(ctr = (64 r + p, j, (REFINE << 28) | tag, i)).
 * ---------------------------------------------------------------------------------- */
enum { STREAM_REFINE = 4, STREAM_MULTINOMIAL = 5 };

uint32_t orc_sweep_uniform(int L, uint64_t seed, uint32_t step, uint32_t slot, int tag, int r, int p)
{
    int hp = 1;
    while (hp < L / 2) hp *= 2;
    uint32_t n = (uint32_t)(r * hp + p);
    uint32_t chunk = n / 32, b = n % 32;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t planes[8];
    for (int call = 0; call < 2; ++call) {
        uint32_t ctr[4] = {2 * chunk + (uint32_t)call, slot,
                           ((uint32_t)STREAM_SWEEP << 28) | (uint32_t)tag, step};
        orc_philox4x32_10(ctr, key, planes + 4 * call);
    }
    uint32_t x = 0;
    for (int k = 0; k < 8; ++k) x |= ((planes[k] >> b) & 1u) << (31 - k);
    uint32_t low = philox_word(seed, (uint32_t)(64 * r + p), slot,
                               ((uint32_t)STREAM_REFINE << 28) | (uint32_t)tag, step, 0);
    return x | (low & 0xFFFFFFu);
}

/* update 0: Metropolis (above); update 1: heatbath (thresholds T_a of
   orc_heatbath_threshold: every site draws its x and flips iff x < T_a). */
void orc_sweep_replica_u(int L, uint64_t seed, uint32_t step, uint32_t slot, double beta,
                         int t0, int theta, int update, int8_t *s)
{
    uint64_t T[5];
    if (update == 1) {
        T[3] = orc_heatbath_threshold(4.0 * beta);
        T[4] = orc_heatbath_threshold(8.0 * beta);
        T[2] = (uint64_t)1 << 31;
        T[1] = ((uint64_t)1 << 32) - T[3];
        T[0] = ((uint64_t)1 << 32) - T[4];
    }
    for (int t = t0; t < t0 + theta; ++t)
        for (int q = 0; q < 2; ++q)
            for (int r = 0; r < L; ++r)
                for (int c = 0; c < L; ++c) {
                    if (((r + c) & 1) != q) continue;
                    int si = s[site(L, r, c)];
                    int a = (s[site(L, r - 1, c)] == si) + (s[site(L, r + 1, c)] == si) +
                            (s[site(L, r, c - 1)] == si) + (s[site(L, r, c + 1)] == si);
                    uint32_t x = orc_sweep_uniform(L, seed, step, slot, 2 * t + q, r, c / 2);
                    int flip;
                    if (update == 1) flip = (uint64_t)x < T[a];
                    else if (a <= 2) flip = 1;
                    else if (a == 3) flip = (uint64_t)x < orc_metropolis_threshold(4.0 * beta);
                    else flip = (uint64_t)x < orc_metropolis_threshold(8.0 * beta);
                    if (flip) s[site(L, r, c)] = (int8_t)(-si);
                }
}

void orc_sweep_replica_t0(int L, uint64_t seed, uint32_t step, uint32_t slot, double beta,
                          int t0, int theta, int8_t *s)
{
    uint64_t T4 = orc_metropolis_threshold(4.0 * beta);
    uint64_t T8 = orc_metropolis_threshold(8.0 * beta);
    for (int t = t0; t < t0 + theta; ++t)
        for (int q = 0; q < 2; ++q)
            for (int r = 0; r < L; ++r)
                for (int c = 0; c < L; ++c) {
                    if (((r + c) & 1) != q) continue;
                    int si = s[site(L, r, c)];
                    int a = (s[site(L, r - 1, c)] == si) + (s[site(L, r + 1, c)] == si) +
                            (s[site(L, r, c - 1)] == si) + (s[site(L, r, c + 1)] == si);
                    uint32_t x = orc_sweep_uniform(L, seed, step, slot, 2 * t + q, r, c / 2);
                    int flip;
                    if (a <= 2) flip = 1;
                    else if (a == 3) flip = (uint64_t)x < T4;
                    else flip = (uint64_t)x < T8;
                    if (flip) s[site(L, r, c)] = (int8_t)(-si);
                }
}

/* Sweeps are numbered from 0 within a temperature step; a run of theta sweeps that starts
   after t0 earlier sweeps of the same step uses sweep numbers t0 .. t0 + theta - 1. */
void orc_sweep_replica(int L, uint64_t seed, uint32_t step, uint32_t slot, double beta,
                       int theta, int8_t *s)
{
    orc_sweep_replica_t0(L, seed, step, slot, beta, 0, theta, s);
}

/* ------------------------------------------------------------------------------------
 * Step 2 (Sec. II): reweighting and resampling from beta_prev to beta_new given the
 * energy levels of the R_prev current replicas (energies BEFORE resampling, as the
 * paper stresses after Eq. boltzmann-weight).
 *   h_k          histogram of levels, E_k = 4k - 2N
 *   E_ref        energy of the lowest occupied level; w_k = exp(-dbeta (E_k - E_ref))
 *   S            sum over occupied k in ascending order of h_k w_k
 *   ln Q_i       = -dbeta E_ref + ln(S / R_prev)          (Eq. Q, shifted by E_ref)
 *   tau_hat_k    = R w_k / S = (R / R_prev) exp(-dbeta E_k) / Q_i   (Eq. taus)
 * Nearest-integer copies (Eq. resampling-factors): with u = x 2^-32 and x word 0 of
 * Philox(ctr = (j, 0, RESAMPLE << 28, i)), r_j = floor(tau) if u > frac(tau), else
 * floor(tau) + 1; equivalently r_j = floor(tau) + [x <= floor(frac(tau) 2^32)].
 * Poisson copies: r_j ~ Poisson(tau_hat) by sequential inversion (see orc_poisson).
 * Children of parent j fill the next r_j slots in parent order (tree order).
 * ---------------------------------------------------------------------------------- */
#define ORC_POISSON_CHUNK 32.0
#define ORC_POISSON_KMAX 1000

/* Poisson(lambda) by inversion of the cumulative distribution (sequential search,
   Devroye 1986, Ch. X.3): u uniform in [0,1) with 53 bits, p_0 = e^{-mu},
   p_k = p_{k-1} mu / k, return the first k with u < F_k.  For lambda >= 32 the draw is
   the sum of m = ceil(lambda / 32) independent Poisson(lambda / m) draws; chunk c uses
   Philox(ctr = (j, c, POISSON << 28, i)), u = (x0 >> 5) 2^-27 + (x1 >> 6) 2^-53. */
int64_t orc_poisson(double lambda, uint64_t seed, uint32_t j, uint32_t step)
{
    if (!(lambda > 0.0)) return 0;
    int64_t m = 1;
    if (lambda >= ORC_POISSON_CHUNK) m = (int64_t)ceil(lambda / ORC_POISSON_CHUNK);
    double mu = lambda / (double)m;
    int64_t total = 0;
    for (int64_t chunk = 0; chunk < m; ++chunk) {
        uint32_t ctr[4] = {j, (uint32_t)chunk, (uint32_t)STREAM_POISSON << 28, step};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        double u = ((double)(out[0] >> 5) * 67108864.0 + (double)(out[1] >> 6)) *
                   (1.0 / 9007199254740992.0);
        double p = orc_exp(-mu);
        double F = p;
        int64_t k = 0;
        while (u >= F && k < ORC_POISSON_KMAX) {
            k = k + 1;
            p = (p * mu) / (double)k;
            F = F + p;
        }
        total += k;
    }
    return total;
}

typedef struct {
    double lnQ;        /* ln Q_i of this step */
    double S;          /* sum_k h_k w_k */
    int32_t kmin;      /* lowest occupied level */
    int32_t pad;
    int64_t R_new;     /* new population size */
} orc_resample_info;

/* A sum in a fixed pairwise order (the reading shared by every level sum of binary64 terms):
   the n terms are cut into 1024 consecutive chunks of ceil(n / 1024) terms, each chunk is
   summed from its first term, and the 1024 chunk sums are added as a binary tree
   (x_j += x_{j + s} for s = 512, 256, ..., 1). */
#define ORC_CHUNKS 1024

static double pairwise_sum(const double *x, int n)
{
    double part[ORC_CHUNKS];
    int c = (n + ORC_CHUNKS - 1) / ORC_CHUNKS;
    for (int j = 0; j < ORC_CHUNKS; ++j) {
        double s = 0.0;
        for (int i = j * c; i < (j + 1) * c && i < n; ++i) s = s + x[i];
        part[j] = s;
    }
    for (int s = ORC_CHUNKS / 2; s > 0; s /= 2)
        for (int j = 0; j < s; ++j) part[j] = part[j] + part[j + s];
    return part[0];
}

/* Step 2's tables from the level histogram h of the R_prev parents (Eqs. Q and taus):
   E_ref = the lowest occupied level's energy, w_k = exp(-dbeta (E_k - E_ref)) for occupied k,
   S = the pairwise sum (above) of h_k w_k over the occupied k, ascending,
   ln Q_i = -dbeta E_ref + ln(S / R_prev),
   tau_k = R_target w_k / S, fl_k = floor(tau_k), thr_k = floor((tau_k - fl_k) 2^32).
   Returns 6 (numeric) for an empty histogram, else 0. */
static int resample_tables(int N, int64_t R_target, const int64_t *h, int64_t R_prev, double dbeta,
                           double *w, double *tau, int64_t *fl, uint64_t *thr, orc_resample_info *info)
{
    int kmin = 0;
    while (kmin <= N && h[kmin] == 0) ++kmin;
    if (kmin > N) return 6;
    int Eref = 4 * kmin - 2 * N;
    for (int k = 0; k <= N; ++k) {
        if (h[k] == 0) continue;
        int Ek = 4 * k - 2 * N;
        w[k] = orc_exp(-(dbeta * (double)(Ek - Eref)));
    }
    double *t = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    int n = 0;
    for (int k = 0; k <= N; ++k)
        if (h[k] != 0) t[n++] = (double)h[k] * w[k];
    double S = pairwise_sum(t, n);
    free(t);
    double lnQ = -(dbeta * (double)Eref) + log(S / (double)R_prev);
    for (int k = 0; k <= N; ++k) {
        if (h[k] == 0) continue;
        tau[k] = ((double)R_target * w[k]) / S;
        double f = floor(tau[k]);
        fl[k] = (int64_t)f;
        thr[k] = (uint64_t)floor((tau[k] - f) * 4294967296.0);
    }
    info->lnQ = lnQ;
    info->S = S;
    info->kmin = kmin;
    return 0;
}

/* Copy number of parent j (global index) at level k (Eq. resampling-factors for nearest
   integer, kind 0; a Poisson draw of mean tau_k, kind 1). */
static int64_t copy_number(int kind, int64_t fl, uint64_t thr, double tau, uint64_t seed, uint32_t j,
                           uint32_t step)
{
    if (kind == 0) {
        uint32_t x = philox_word(seed, j, 0, (uint32_t)STREAM_RESAMPLE << 28, step, 0);
        return fl + (((uint64_t)x <= thr) ? 1 : 0);
    }
    return orc_poisson(tau, seed, j, step);
}

/* Status codes shared in meaning (not in code) with the library: 0 ok, 3 capacity,
   6 numeric (empty population). */
int orc_resample_levels(int L, int64_t R_target, int64_t R_prev, const int32_t *level,
                        double beta_prev, double beta_new, uint32_t step, uint64_t seed,
                        int kind, int64_t capacity, int32_t *counts_out,
                        orc_resample_info *info)
{
    int N = L * L;
    int64_t *h = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    double *w = (double *)calloc((size_t)N + 1, sizeof(double));
    double *tau = (double *)calloc((size_t)N + 1, sizeof(double));
    int64_t *fl = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    uint64_t *thr = (uint64_t *)calloc((size_t)N + 1, sizeof(uint64_t));
    for (int64_t j = 0; j < R_prev; ++j) h[level[j]] += 1;
    double dbeta = beta_new - beta_prev;
    if (resample_tables(N, R_target, h, R_prev, dbeta, w, tau, fl, thr, info) != 0) {
        free(h); free(w); free(tau); free(fl); free(thr);
        return 6;
    }
    int64_t R_new = 0;
    if (kind == 2) {
        /* Multinomial resampling at fixed size (Sec. II: R_target children drawn from the
           parents with probabilities tau_j / R_prev = w_j / sum_l w_l).  Reading: the weights
           are the integers W_j = floor(w_{k(j)} 2^32) (w <= 1), C_j = W_0 + ... + W_j exactly,
           T = C_{R_prev - 1}; child c takes X = x1 2^32 + x0 from words 0 and 1 of
           Philox(ctr = (c, 0, MULTINOMIAL << 28, i)), U = floor(X T / 2^64) in [0, T), and
           the parent j with C_{j-1} <= U < C_j.  counts_out[j] = children of parent j. */
        uint64_t *C = (uint64_t *)malloc((size_t)R_prev * sizeof(uint64_t));
        uint64_t run = 0;
        for (int64_t j = 0; j < R_prev; ++j) {
            run += (uint64_t)floor(w[level[j]] * 4294967296.0);
            C[j] = run;
            counts_out[j] = 0;
        }
        const uint64_t T = run;
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (int64_t c = 0; c < R_target; ++c) {
            uint32_t ctr[4] = {(uint32_t)c, 0, (uint32_t)STREAM_MULTINOMIAL << 28, step}, x[4];
            orc_philox4x32_10(ctr, key, x);
            const uint64_t X = ((uint64_t)x[1] << 32) | x[0];
            const uint64_t U = (uint64_t)(((unsigned __int128)X * T) >> 64);
            int64_t lo = 0, hi = R_prev - 1;  /* first j with C_j > U */
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (C[mid] > U) hi = mid;
                else lo = mid + 1;
            }
            counts_out[lo] += 1;
        }
        free(C);
        R_new = R_target;
    }
    for (int64_t j = 0; kind != 2 && j < R_prev; ++j) {
        int k = level[j];
        int64_t r = copy_number(kind, fl[k], thr[k], tau[k], seed, (uint32_t)j, step);
        counts_out[j] = (int32_t)r;
        R_new += r;
    }
    info->R_new = R_new;
    free(h); free(w); free(tau); free(fl); free(thr);
    if (R_new > capacity) return 3;
    if (R_new == 0) return 6;
    return 0;
}

/* Copy numbers of the n parents of one shard of a population split by contiguous slot
   ranges (a population too large for one device): h is the level histogram of the whole
   population of R_prev parents, so the tables (and ln Q_i) are those of the whole
   population, and local parent j has the global index parent_base + j, which keys its
   random numbers.  Every shard thus draws the numbers one unsplit population would draw.
   Nearest-integer (kind 0) and Poisson (kind 1) need nothing else.  Multinomial (kind 2)
   also needs h_before, the level histogram of the parents at global indices below
   parent_base (the shards before this one): with the integer weights W_k of the whole
   population's table, the running sum of the weights at this shard's first parent is
   B = sum_k h_before_k W_k and the total is T = sum_k h_k W_k (exact integers, so the same as
   summing parent by parent); every child c of the whole population draws its U as in
   orc_resample_levels, and those with B <= U < B + (this shard's weight sum) land on one of
   this shard's parents, found in the shard's own running sums.  info->R_new = this shard's
   children; 6 for an empty histogram, 1 for an unknown kind or a missing h_before. */
int orc_resample_shard(int L, int64_t R_target, const int64_t *h, int64_t R_prev, int64_t n,
                       const int32_t *level, int64_t parent_base, double beta_prev, double beta_new,
                       uint32_t step, uint64_t seed, int kind, const int64_t *h_before, int32_t *counts_out,
                       orc_resample_info *info)
{
    if (kind != 0 && kind != 1 && kind != 2) return 1;
    if (kind == 2 && !h_before) return 1;
    int N = L * L;
    double *w = (double *)calloc((size_t)N + 1, sizeof(double));
    double *tau = (double *)calloc((size_t)N + 1, sizeof(double));
    int64_t *fl = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    uint64_t *thr = (uint64_t *)calloc((size_t)N + 1, sizeof(uint64_t));
    int st = resample_tables(N, R_target, h, R_prev, beta_new - beta_prev, w, tau, fl, thr, info);
    int64_t R_new = 0;
    if (st == 0 && kind == 2) {
        uint64_t T = 0, B = 0;
        for (int k = 0; k <= N; ++k) {
            if (h[k] == 0) continue;
            const uint64_t Wk = (uint64_t)floor(w[k] * 4294967296.0);
            T += (uint64_t)h[k] * Wk;
            B += (uint64_t)h_before[k] * Wk;
        }
        uint64_t *C = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
        uint64_t run = B;
        for (int64_t j = 0; j < n; ++j) {
            run += (uint64_t)floor(w[level[j]] * 4294967296.0);
            C[j] = run;
            counts_out[j] = 0;
        }
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (int64_t c = 0; n > 0 && c < R_target; ++c) {
            uint32_t ctr[4] = {(uint32_t)c, 0, (uint32_t)STREAM_MULTINOMIAL << 28, step}, x[4];
            orc_philox4x32_10(ctr, key, x);
            const uint64_t X = ((uint64_t)x[1] << 32) | x[0];
            const uint64_t U = (uint64_t)(((unsigned __int128)X * T) >> 64);
            if (U < B || U >= C[n - 1]) continue;  /* a parent of another shard */
            int64_t lo = 0, hi = n - 1;  /* first local j with C_j > U */
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (C[mid] > U) hi = mid;
                else lo = mid + 1;
            }
            counts_out[lo] += 1;
            R_new += 1;
        }
        free(C);
    }
    for (int64_t j = 0; st == 0 && kind != 2 && j < n; ++j) {
        int k = level[j];
        int64_t r = copy_number(kind, fl[k], thr[k], tau[k], seed, (uint32_t)(parent_base + j), step);
        counts_out[j] = (int32_t)r;
        R_new += r;
    }
    info->R_new = R_new;
    free(w); free(tau); free(fl); free(thr);
    return st;
}

/* ------------------------------------------------------------------------------------
 * The population: a full PA run held on the host.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int L, N, kind;
    int update;             /* 0 Metropolis, 1 heatbath */
    int64_t R_target, capacity, R;
    uint64_t seed;
    uint32_t step;          /* index i of the current temperature beta_i */
    double beta, dbeta, lnQ, sum_lnQ;
    double sum_lnR;         /* sum_k ln(R_{k-1} / R) over the resamplings so far */
    int theta_last;
    int t_done;             /* sweeps already done at the current step */
    int8_t *s;              /* capacity * N */
    int8_t *s_next;
    int32_t *E, *M, *fam, *E_next, *M_next, *fam_next;
    int32_t *counts;        /* copy numbers of the last resampling, R_prev entries */
    int64_t R_prev;
    int status;
} orc_pa;

void orc_pa_destroy(orc_pa *p);

orc_pa *orc_pa_create(int L, int64_t R, int64_t capacity, uint64_t seed, int kind)
{
    if (L < 4 || (L % 2) != 0 || L > 128 || R < 1 || capacity < R) return NULL;
    orc_pa *p = (orc_pa *)calloc(1, sizeof(orc_pa));
    p->L = L; p->N = L * L; p->kind = kind;
    p->R_target = R; p->capacity = capacity; p->seed = seed;
    size_t cap = (size_t)capacity;
    p->s = (int8_t *)malloc(cap * (size_t)p->N);
    p->s_next = (int8_t *)malloc(cap * (size_t)p->N);
    p->E = (int32_t *)malloc(cap * 4); p->M = (int32_t *)malloc(cap * 4);
    p->fam = (int32_t *)malloc(cap * 4);
    p->E_next = (int32_t *)malloc(cap * 4); p->M_next = (int32_t *)malloc(cap * 4);
    p->fam_next = (int32_t *)malloc(cap * 4);
    p->counts = (int32_t *)malloc(cap * 4);
    if (!p->s || !p->s_next || !p->E || !p->M || !p->fam || !p->E_next || !p->M_next ||
        !p->fam_next || !p->counts) {
        orc_pa_destroy(p);
        return NULL;
    }
    return p;
}

void orc_pa_destroy(orc_pa *p)
{
    if (!p) return;
    free(p->s); free(p->s_next); free(p->E); free(p->M); free(p->fam);
    free(p->E_next); free(p->M_next); free(p->fam_next); free(p->counts);
    free(p);
}

static void measure_all(orc_pa *p)
{
    for (int64_t j = 0; j < p->R; ++j)
        orc_energy_mag(p->L, p->s + (size_t)j * p->N, &p->E[j], &p->M[j]);
}

/* Step 1: R_0 = R replicas by simple sampling at beta_0 = 0, family id = own index. */
void orc_pa_init(orc_pa *p)
{
    p->R = p->R_target;
    p->R_prev = 0;
    p->step = 0;
    p->beta = 0.0; p->dbeta = 0.0; p->lnQ = 0.0; p->sum_lnQ = 0.0; p->sum_lnR = 0.0;
    p->theta_last = 0;
    p->t_done = 0;
    p->status = 0;
    for (int64_t j = 0; j < p->R; ++j) {
        orc_init_replica(p->L, p->seed, (uint32_t)j, p->s + (size_t)j * p->N);
        p->fam[j] = (int32_t)j;
    }
    measure_all(p);
}

/* Step 2: resample from the current beta to beta_new; step index advances by one. */
int orc_pa_resample(orc_pa *p, double beta_new)
{
    if (p->status) return p->status;
    int N = p->N;
    int32_t *level = (int32_t *)malloc((size_t)p->R * 4);
    for (int64_t j = 0; j < p->R; ++j) level[j] = (p->E[j] + 2 * N) / 4;
    orc_resample_info info;
    uint32_t step = p->step + 1;
    int st = orc_resample_levels(p->L, p->R_target, p->R, level, p->beta, beta_new, step,
                                 p->seed, p->kind, p->capacity, p->counts, &info);
    free(level);
    if (st) { p->status = st; return st; }
    int64_t slot = 0;
    for (int64_t j = 0; j < p->R; ++j)
        for (int32_t c = 0; c < p->counts[j]; ++c) {
            memcpy(p->s_next + (size_t)slot * N, p->s + (size_t)j * N, (size_t)N);
            p->E_next[slot] = p->E[j];
            p->M_next[slot] = p->M[j];
            p->fam_next[slot] = p->fam[j];
            ++slot;
        }
    int8_t *ts = p->s; p->s = p->s_next; p->s_next = ts;
    int32_t *t;
    t = p->E; p->E = p->E_next; p->E_next = t;
    t = p->M; p->M = p->M_next; p->M_next = t;
    t = p->fam; p->fam = p->fam_next; p->fam_next = t;
    p->R_prev = p->R;
    p->R = info.R_new;
    p->dbeta = beta_new - p->beta;
    p->beta = beta_new;
    p->step = step;
    p->t_done = 0;
    p->lnQ = info.lnQ;
    p->sum_lnQ = p->sum_lnQ + info.lnQ;
    p->sum_lnR = p->sum_lnR + log((double)p->R_prev / (double)p->R_target);
    return 0;
}

/* Step 3 then the measurement of step 4: theta sweeps of every replica at the current
   beta, then energies and magnetisations. */
void orc_pa_set_update(orc_pa *p, int update) { p->update = update; }

void orc_pa_sweep(orc_pa *p, int theta)
{
    for (int64_t j = 0; j < p->R; ++j)
        orc_sweep_replica_u(p->L, p->seed, p->step, (uint32_t)j, p->beta, p->t_done, theta, p->update,
                            p->s + (size_t)j * p->N);
    p->t_done += theta;
    p->theta_last = theta;
    measure_all(p);
}

/* Step 4: population averages (Sec. III) and the free energy (Sec. VII) of a population of
   R replicas, from its exact integer sums; formula order fixed.
   isums[0] sum E, [1] sum E^2, [2] sum |M|, [3] sum M^2, [4] families f, [5] sum size^2.
   out[0] beta, [1] dbeta, [2] R_i, [3] e, [4] C, [5] m, [6] m2, [7] chi, [8] lnQ,
   [9] -beta F, [10] families f, [11] rho_t, [12] step, [13] theta,
   [14] sum_k ln(R_{k-1} / R) (the population-size factor of Eq. modified-weights2). */
void orc_observables_from_sums(int N, int64_t R, const int64_t *isums, double beta, double dbeta,
                               double lnQ, double sum_lnQ, double sum_lnR, uint32_t step, int theta,
                               double *out)
{
    double Rd = (double)R, Nd = (double)N, b = beta;
    double meanE = (double)isums[0] / Rd;
    double meanE2 = (double)isums[1] / Rd;
    double e = meanE / Nd;
    double C = ((b * b) * (meanE2 - meanE * meanE)) / Nd;
    double m = ((double)isums[2] / Rd) / Nd;
    double m2 = ((double)isums[3] / Rd) / (Nd * Nd);
    double chi = (b * Nd) * (m2 - m * m);
    double rho_t = (double)isums[5] / Rd;
    double mbF = Nd * 0.6931471805599453094 + sum_lnQ;
    out[0] = beta; out[1] = dbeta; out[2] = Rd; out[3] = e; out[4] = C;
    out[5] = m; out[6] = m2; out[7] = chi; out[8] = lnQ; out[9] = mbF;
    out[10] = (double)isums[4]; out[11] = rho_t; out[12] = (double)step;
    out[13] = (double)theta;
    out[14] = sum_lnR;
}

/* The exact integer sums of the current population (isums as above): energies and
   magnetisations summed over replicas; families (Sec. V) are the runs of equal ids, which
   stay sorted in tree order. */
void orc_population_sums(int64_t R, const int32_t *E, const int32_t *M, const int32_t *fam, int64_t *isums)
{
    int64_t sE = 0, sE2 = 0, sAM = 0, sM2 = 0;
    for (int64_t j = 0; j < R; ++j) {
        int64_t e = E[j], m = M[j];
        sE += e; sE2 += e * e;
        sAM += (m < 0 ? -m : m);
        sM2 += m * m;
    }
    int64_t f = 0, s2 = 0, run = 0;
    for (int64_t j = 0; j < R; ++j) {
        if (j == 0 || fam[j] != fam[j - 1]) {
            if (run) s2 += run * run;
            run = 0;
            ++f;
        }
        ++run;
    }
    if (run) s2 += run * run;
    isums[0] = sE; isums[1] = sE2; isums[2] = sAM; isums[3] = sM2; isums[4] = f; isums[5] = s2;
}

void orc_pa_observables(const orc_pa *p, double *out, int64_t *isums)
{
    int64_t sums[6];
    orc_population_sums(p->R, p->E, p->M, p->fam, sums);
    orc_observables_from_sums(p->N, p->R, sums, p->beta, p->dbeta, p->lnQ, p->sum_lnQ, p->sum_lnR, p->step,
                              p->theta_last, out);
    if (isums) memcpy(isums, sums, sizeof(sums));
}

/* ------------------------------------------------------------------------------------
 * Adaptive temperature step (the paper names it, Sec. II and Sec. IX, and recommends a
 * step that keeps the energy-histogram overlap above about 0.7, Sec. X; the procedure itself
 * is not printed).  Reading: the overlap of the energy distribution at beta, estimated by
 * the population histogram p_k = h_k / R, with the one reweighted to beta + dbeta,
 * q_k = t_k / S, t_k = h_k w_k, w_k = exp(-dbeta (E_k - E_ref)) (E_ref as in the resampling
 * step), S = sum of the t_k, is
 *     alpha(dbeta) = sum over occupied k of min(p_k, q_k).
 * Both sums run over the occupied levels in ascending order, in a fixed pairwise order: the
 * n terms are cut into 1024 consecutive chunks of c = ceil(n / 1024) terms, each chunk is
 * summed from its first term, and the 1024 chunk sums are added as a binary tree
 * (x_i = x_i + x_{i+s} for s = 512, 256, ..., 1; result x_0).
 * The next step is the largest dbeta in (0, hi], hi = min(dbeta_max, beta_final - beta),
 * with alpha(dbeta) >= alpha_target: hi itself if it qualifies; else a search keeps a
 * bracket [lo, hi) with alpha(lo) >= alpha_target (lo = 0 at first) and, ceil(iters / 6)
 * times, evaluates the K - 1 = 63 points x_m = lo + (hi - lo) (m / 64), takes m* = the
 * number of leading points that reach the target and narrows the bracket to
 * [x_{m*}, x_{m*+1}) (x_0 = lo, x_64 = hi).  If no point ever qualifies, the step is the
 * smallest tried (the final hi).
 * ---------------------------------------------------------------------------------- */
#define ORC_SEARCH_K 64

double orc_overlap(int N, const int64_t *h, double dbeta)
{
    int kmin = 0;
    while (kmin <= N && h[kmin] == 0) ++kmin;
    if (kmin > N) return 0.0;
    int Eref = 4 * kmin - 2 * N;
    int64_t R = 0;
    for (int k = 0; k <= N; ++k) R += h[k];
    double *t = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *m = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    int *occ = (int *)malloc(sizeof(int) * (size_t)(N + 1));
    int n = 0;
    for (int k = 0; k <= N; ++k)
        if (h[k] != 0) occ[n++] = k;
    for (int i = 0; i < n; ++i) {
        int k = occ[i];
        double w = orc_exp(-(dbeta * (double)(4 * k - 2 * N - Eref)));
        t[i] = (double)h[k] * w;
    }
    double S = pairwise_sum(t, n);
    /* p_k = h_k (1 / R), q_k = t_k (1 / S): the reciprocals formed once */
    const double invR = 1.0 / (double)R, invS = 1.0 / S;
    for (int i = 0; i < n; ++i) {
        double pk = (double)h[occ[i]] * invR;
        double qk = t[i] * invS;
        m[i] = pk < qk ? pk : qk;
    }
    double alpha = pairwise_sum(m, n);
    free(t); free(m); free(occ);
    return alpha;
}

double orc_bisect_next_beta(int N, const int64_t *h, double beta, double beta_final, double dbeta_max,
                            double alpha_target, int iters, double *alpha_out)
{
    double hi = beta_final - beta;
    if (dbeta_max < hi) hi = dbeta_max;
    if (!(hi > 0.0)) {
        if (alpha_out) *alpha_out = 1.0;
        return beta_final;
    }
    const double hi0 = hi;
    double dbeta, alpha;
    double a_hi = orc_overlap(N, h, hi);
    if (a_hi >= alpha_target) {
        dbeta = hi;
        alpha = a_hi;
    } else {
        double lo = 0.0, a_lo = 1.0;
        const int rounds = (iters + 5) / 6;
        for (int r = 0; r < rounds; ++r) {
            const double d = hi - lo;
            double a[ORC_SEARCH_K];
            for (int j = 1; j < ORC_SEARCH_K; ++j)
                a[j] = orc_overlap(N, h, lo + d * ((double)j / (double)ORC_SEARCH_K));
            int ms = 0;
            while (ms + 1 < ORC_SEARCH_K && a[ms + 1] >= alpha_target) ++ms;
            const double new_lo = lo + d * ((double)ms / (double)ORC_SEARCH_K);
            const double new_hi = lo + d * ((double)(ms + 1) / (double)ORC_SEARCH_K);
            if (ms > 0) {
                lo = new_lo;
                a_lo = a[ms];
            }
            if (ms + 1 < ORC_SEARCH_K) hi = new_hi;
        }
        if (lo > 0.0) {
            dbeta = lo;
            alpha = a_lo;
        } else { /* no tried step reaches the target: take the smallest one tried */
            dbeta = hi;
            alpha = orc_overlap(N, h, hi);
        }
    }
    if (alpha_out) *alpha_out = alpha;
    if (dbeta == hi0 && hi0 == beta_final - beta) return beta_final;
    return beta + dbeta;
}

/* A proposed step (from the learned schedule) is kept if the overlap at that step reaches
   alpha_floor (the proposal is first clipped to hi); otherwise the bisection above decides.
   *source: 2 = proposal kept, 3 = bisection fallback. */
double orc_accept_or_bisect(int N, const int64_t *h, double beta, double beta_final, double dbeta_max,
                            double dbeta_prop, double alpha_floor, double alpha_target, int iters,
                            double *alpha_out, int *source)
{
    double hi = beta_final - beta;
    if (dbeta_max < hi) hi = dbeta_max;
    if (!(hi > 0.0)) {
        if (alpha_out) *alpha_out = 1.0;
        *source = 2;
        return beta_final;
    }
    double dp = dbeta_prop;
    if (dp > hi) dp = hi;
    double a_p = orc_overlap(N, h, dp);
    if (a_p >= alpha_floor) {
        if (alpha_out) *alpha_out = a_p;
        *source = 2;
        if (dp == hi && hi == beta_final - beta) return beta_final;
        return beta + dp;
    }
    *source = 3;
    return orc_bisect_next_beta(N, h, beta, beta_final, dbeta_max, alpha_target, iters, alpha_out);
}

double orc_pa_propose_bisect(const orc_pa *p, double beta_final, double dbeta_max, double alpha_target,
                             int iters, double *alpha_out)
{
    int64_t *h = (int64_t *)calloc((size_t)p->N + 1, sizeof(int64_t));
    for (int64_t j = 0; j < p->R; ++j) h[(p->E[j] + 2 * p->N) / 4] += 1;
    double b = orc_bisect_next_beta(p->N, h, p->beta, beta_final, dbeta_max, alpha_target, iters, alpha_out);
    free(h);
    return b;
}

/* Accessors used by the tests. */
int64_t orc_pa_R(const orc_pa *p) { return p->R; }
int64_t orc_pa_R_prev(const orc_pa *p) { return p->R_prev; }
int orc_pa_status(const orc_pa *p) { return p->status; }
double orc_pa_sum_lnQ(const orc_pa *p) { return p->sum_lnQ; }

void orc_pa_histogram(const orc_pa *p, int32_t *h)
{
    memset(h, 0, sizeof(int32_t) * (size_t)(p->N + 1));
    for (int64_t j = 0; j < p->R; ++j) h[(p->E[j] + 2 * p->N) / 4] += 1;
}

void orc_pa_hashes(const orc_pa *p, uint64_t *out)
{
    for (int64_t j = 0; j < p->R; ++j) out[j] = orc_hash(p->L, p->s + (size_t)j * p->N);
}

void orc_pa_get(const orc_pa *p, int32_t *E, int32_t *M, int32_t *fam)
{
    for (int64_t j = 0; j < p->R; ++j) {
        if (E) E[j] = p->E[j];
        if (M) M[j] = p->M[j];
        if (fam) fam[j] = p->fam[j];
    }
}

void orc_pa_counts(const orc_pa *p, int32_t *out)
{
    for (int64_t j = 0; j < p->R_prev; ++j) out[j] = p->counts[j];
}

void orc_pa_spins(const orc_pa *p, int64_t first, int64_t count, int8_t *out)
{
    memcpy(out, p->s + (size_t)first * p->N, (size_t)count * p->N);
}

/* Replace the population (for stepwise replay from an externally produced state). */
int orc_pa_set(orc_pa *p, int64_t R, const int8_t *spins, const int32_t *fam,
               uint32_t step, double beta, double sum_lnQ)
{
    if (R < 1 || R > p->capacity) return 1;
    p->R = R;
    memcpy(p->s, spins, (size_t)R * p->N);
    for (int64_t j = 0; j < R; ++j) p->fam[j] = fam[j];
    p->step = step;
    p->beta = beta;
    p->sum_lnQ = sum_lnQ;
    p->t_done = 0;
    p->status = 0;
    measure_all(p);
    return 0;
}

/* Population analysis of the current population (blocked and jackknife errors, effective
   population sizes, family entropy): see pa_analysis.c. */
int orc_analysis(int N, double beta, int64_t R, const int32_t *E, const int32_t *M, const int32_t *fam,
                 int n, double *out);

int orc_pa_analysis(const orc_pa *p, int n, double *out)
{
    return orc_analysis(p->N, p->beta, p->R, p->E, p->M, p->fam, n, out);
}

/* ------------------------------------------------------------------------------------
 * Weighted averages over M independent runs at the same temperature step (Sec. VIII,
 * Eqs. weighted-averages and modified-weights2).  Run m has population R_i^m, target R^m,
 * -beta F^m = N ln 2 + sum_k ln Q_k^m and s^m = sum_{k<=i} ln(R_{k-1}^m / R^m):
 *   log w_m = ln R_i^m - beta F^m (+ s^m for mode 1, the fluctuating-size form),
 *   omega_m = exp(log w_m - max) / sum_l exp(log w_l - max)      (runs in order),
 *   O = sum_m omega_m O_m for O in (e, C, m, m2, chi), and the plain means (1/M) sum_m O_m.
 * Also M_eff = 1 / sum omega_m^2, the largest omega, the unbiased variance of -beta F^m over
 * the runs (weighted averaging is sound only while it is well below 1, Sec. VIII), and the
 * combined free energy ln(sum_m R^m exp(-beta F^m) / sum_m R^m) (reading: the R-weighted
 * mean of the runs' partition-function estimates).
 * obs is M x 5 (e, C, m, m2, chi).  out: [0] M_eff, [1] max omega, [2] var(-beta F),
 * [3] combined -beta F, [4..8] weighted e C m m2 chi, [9..13] plain means. */
void orc_weighted_average(int M, const double *R_i, const double *R_t, const double *mbF, const double *slnR,
                          const double *obs, int mode, double *out)
{
    double mx = -INFINITY, mz = -INFINITY, sR = 0.0;
    for (int m = 0; m < M; ++m) {
        const double lw = log(R_i[m]) + mbF[m] + (mode == 1 ? slnR[m] : 0.0);
        const double lz = log(R_t[m]) + mbF[m];
        if (lw > mx) mx = lw;
        if (lz > mz) mz = lz;
        sR += R_t[m];
    }
    double s = 0.0, sz = 0.0;
    for (int m = 0; m < M; ++m) {
        s += exp(log(R_i[m]) + mbF[m] + (mode == 1 ? slnR[m] : 0.0) - mx);
        sz += exp(log(R_t[m]) + mbF[m] - mz);
    }
    double w2 = 0.0, wmax = 0.0, meanF = 0.0;
    for (int q = 0; q < 5; ++q) { out[4 + q] = 0.0; out[9 + q] = 0.0; }
    for (int m = 0; m < M; ++m) {
        const double om = exp(log(R_i[m]) + mbF[m] + (mode == 1 ? slnR[m] : 0.0) - mx) / s;
        w2 += om * om;
        if (om > wmax) wmax = om;
        for (int q = 0; q < 5; ++q) {
            out[4 + q] += om * obs[5 * m + q];
            out[9 + q] += obs[5 * m + q];
        }
        meanF += mbF[m];
    }
    meanF /= (double)M;
    double vF = 0.0;
    for (int m = 0; m < M; ++m) vF += (mbF[m] - meanF) * (mbF[m] - meanF);
    vF = M > 1 ? vF / (double)(M - 1) : 0.0;
    for (int q = 0; q < 5; ++q) out[9 + q] /= (double)M;
    out[0] = 1.0 / w2;
    out[1] = wmax;
    out[2] = vF;
    out[3] = mz + log(sz) - log(sR);
}
