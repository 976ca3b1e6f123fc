/*
 * qed_oracle.c -- plain FP64 CPU oracle for the spin- and polarization-resolved
 * strong-field QED particle step of Qian, Seipt, Vranic, Grismayer, Ridgers and
 * Thomas, "A Fully Spin and Polarization Resolved Strong Field QED Algorithm for
 * Particle-in-Cell Codes" (arXiv:2511.08929).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Conventions (the readings of the paper are listed in the design notes):
 *   units: time 1/omega, length c/omega, momentum m c, fields m c omega / e,
 *          charge q = -1 (electron), +1 (positron), photon energy in m c^2.
 *   eta0 = hbar omega / (m c^2); the Schwinger field is 1/eta0 in these units.
 *
 * Every function cites the section / equation of the paper it restates.
 * Everything is double precision, no FMA contraction (built with
 * -ffp-contract=off), loops over particles are the only parallelism (OpenMP).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_ALPHA 7.2973525693e-3 /* fine-structure constant (CODATA 2018) */
#define ORC_SQRT3 1.73205080756887729353

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):  */
/* 10 rounds; each round multiplies words 0 and 2 by the two round constants, */
/* mixes high halves with words 1, 3 and the key; the key is bumped by the    */
/* two Weyl constants between rounds.                                         */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in the open interval (0,1) from two 32-bit words: 52 random bits
 * m = (hi >> 12) * 2^32 + lo, u = (m + 1/2) * 2^-52 (exact in double). */
double orc_uniform(uint32_t hi, uint32_t lo)
{
    uint64_t m = ((uint64_t)(hi >> 12) << 32) | (uint64_t)lo;
    return ((double)m + 0.5) * 0x1.0p-52;
}

/* The method's random draws are keyed by (particle id, step, slot):
 * key = (id ^ seed), counter = (step_lo, step_hi, slot, 0).  One Philox call
 * gives four words = two uniforms (words 0,1 and words 2,3). */
void orc_draw(uint64_t id, uint64_t seed, uint64_t step, uint32_t slot, uint32_t out[4])
{
    uint64_t k = id ^ seed;
    uint32_t key[2] = {(uint32_t)k, (uint32_t)(k >> 32)};
    uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(step >> 32), slot, 0u};
    orc_philox4x32_10(ctr, key, out);
}

void orc_uniform_pair(uint64_t id, uint64_t seed, uint64_t step, uint32_t slot, double u[2])
{
    uint32_t w[4];
    orc_draw(id, seed, step, slot, w);
    u[0] = orc_uniform(w[0], w[1]);
    u[1] = orc_uniform(w[2], w[3]);
}

/* Reserved step value for a particle's first optical-depth draw. */
#define ORC_STEP_BIRTH 0xFFFFFFFFFFFFFFFFull
/* Draw slots. */
#define ORC_SLOT_TAU_BRANCH 0u /* u0: optical depth (or r1 in probability mode), u1: branch r_b */
#define ORC_SLOT_LAMBDA_SPIN 1u /* u0: r2 (energy fraction), u1: r3 (spin collapse) */
#define ORC_SLOT_STOKES 2u      /* u0: r4 (Stokes collapse) */
#define ORC_SLOT_CHILD 3u       /* words 0,1: first daughter id, words 2,3: second daughter id */

/* Optical depth a particle starts with: tau = -ln u (Sec. 4.1, optical-depth method). */
double orc_birth_tau(uint64_t id, uint64_t seed)
{
    double u[2];
    orc_uniform_pair(id, seed, ORC_STEP_BIRTH, ORC_SLOT_TAU_BRANCH, u);
    return -log(u[0]);
}

void orc_child_ids(uint64_t id, uint64_t seed, uint64_t step, uint64_t out[2])
{
    uint32_t w[4];
    orc_draw(id, seed, step, ORC_SLOT_CHILD, w);
    out[0] = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    out[1] = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
}

/* ------------------------------------------------------------------------- */
/* Modified Bessel functions (the Bessel form of the spectra, App. A uses      */
/* K_{1/3}, K_{2/3} and IntK_{1/3}(x) = int_x^inf K_{1/3}).                    */
/* Integral representation (DLMF 10.32.9):                                     */
/*   e^x K_nu(x)        = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt           */
/*   e^x IntK_{1/3}(x)  = int_0^inf exp(-x (cosh t - 1)) cosh(t/3) / cosh t dt   */
/* (the second by integrating the first over x).  Trapezoid rule on [0, T],    */
/* step halved until two successive results agree to 1e-15.                    */
/* out = {e^x K13, e^x K23, e^x IntK13}; x > 0.                                 */
/* ------------------------------------------------------------------------- */
static void trap_terms(double x, double t, double w, double acc[3])
{
    double ch = cosh(t), c3 = cosh(t / 3.0), sh = sinh(0.5 * t);
    double e = exp(-x * (2.0 * sh * sh)) * w; /* cosh t - 1 = 2 sinh^2(t/2), no cancellation */
    acc[0] += e * c3;
    acc[1] += e * (2.0 * c3 * c3 - 1.0); /* cosh(2t/3) = 2 cosh^2(t/3) - 1 */
    acc[2] += e * c3 / ch;
}

void orc_bessel_scaled(double x, double out[3])
{
    if (!(x > 0.0)) {
        out[0] = out[1] = INFINITY;
        out[2] = ORC_PI / ORC_SQRT3; /* int_0^inf K_{1/3} = pi/(2 cos(pi/6)) */
        return;
    }
    /* truncation point: integrand below e^-46 times its value at t = 0; the
     * starting step is a quarter of it, so the node count follows the width of the integrand */
    double T = acosh(1.0 + 46.0 / x);
    while (x * (cosh(T) - 1.0) - (2.0 / 3.0) * T < 46.0 && T < 400.0) T += 0.125;
    double h = T / 4.0;
    long n = 4; /* nodes t_m = m h, m = 0..n */
    double sum[3] = {0, 0, 0};
    trap_terms(x, 0.0, 0.5, sum);
    for (long m = 1; m <= n; ++m) trap_terms(x, m * h, 1.0, sum);
    double prev[3] = {sum[0] * h, sum[1] * h, sum[2] * h};
    for (int level = 1; level < 16; ++level) {
        /* halve the step: add the midpoints t = (2m - 1) h/2 */
        double hn = h / 2.0;
        for (long m = 1; m <= n; ++m) trap_terms(x, (2 * m - 1) * hn, 1.0, sum);
        h = hn;
        n *= 2;
        double cur[3] = {sum[0] * h, sum[1] * h, sum[2] * h};
        int done = level >= 3;
        for (int i = 0; i < 3; ++i)
            if (fabs(cur[i] - prev[i]) > 4e-15 * fabs(cur[i])) done = 0;
        for (int i = 0; i < 3; ++i) prev[i] = cur[i];
        if (done) break;
    }
    out[0] = prev[0];
    out[1] = prev[1];
    out[2] = prev[2];
}

/* Unscaled values, for tests and rate integrals. */
void orc_bessel(double x, double out[3])
{
    orc_bessel_scaled(x, out);
    double e = exp(-x);
    out[0] *= e;
    out[1] *= e;
    out[2] *= e;
}

/* ------------------------------------------------------------------------- */
/* Small vector helpers                                                       */
/* ------------------------------------------------------------------------- */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3])
{
    double c0 = a[1] * b[2] - a[2] * b[1];
    double c1 = a[2] * b[0] - a[0] * b[2];
    double c2 = a[0] * b[1] - a[1] * b[0];
    c[0] = c0; c[1] = c1; c[2] = c2;
}

/* ------------------------------------------------------------------------- */
/* Spin- and polarization-resolved spectra, Appendix A (Bessel forms).          */
/* The basis is (eps, beta, k), right-handed: beta = k x eps.                  */
/* All spectra are returned "ignoring the common constant" as the paper does;  */
/* `scale` multiplies the Bessel values (1 for the physical spectrum, e^{u'}    */
/* for scaled values whose ratios are the same).                              */
/* ------------------------------------------------------------------------- */

/* NLC, Eq. (w) of App. A.1 (and Sec. 3.1):
 *   w = -IntK13(u') + kappa K23(u') + lambda (s_i . beta) K13(u'),
 *   g = u K13 beta + (-IntK13 + 2 K23) s_i + lambda u (-IntK13 + K23)(s_i . k) k,
 * with u = lambda/(1-lambda), u' = 2u/(3 chi), kappa = 1/(1-lambda) + (1-lambda).
 * bes = {K13, K23, IntK13} at u' (any common scale). */
void orc_nlc_wg(double lam, const double bes[3], const double si[3], const double eps[3],
                const double beta[3], const double k[3], double *w, double g[3])
{
    double one_m = 1.0 - lam;
    double u = lam / one_m;
    double kappa = 1.0 / one_m + one_m;
    double K13 = bes[0], K23 = bes[1], IK = bes[2];
    (void)eps;
    double sb = dot3(si, beta), sk = dot3(si, k);
    *w = -IK + kappa * K23 + lam * sb * K13;
    double cb = u * K13, cs = -IK + 2.0 * K23, ck = lam * u * (-IK + K23) * sk;
    for (int i = 0; i < 3; ++i) g[i] = cb * beta[i] + cs * si[i] + ck * k[i];
}

/* NLC photon Stokes spectrum, App. A.1: F = F0 + xi . F with
 *   F0 = w + s_f . g                                         (Eq. F0 rearranged)
 *   F1 = -K13 (u (s_i.eps) + lambda (s_f.eps))
 *        - (lambda u / 2) IntK13 ((s_f.eps)(s_i.beta) + (s_f.beta)(s_i.eps))
 *        + (kappa~/2) K23 (s_f x s_i) . k                                  (Eq. F1)
 *   F2 = (kappa~/2) K13 (s_f x s_i) . eps - (lambda IntK13 - kappa~ K23)(s_i.k)
 *        - (u IntK13 - kappa~ K23)(s_f.k)
 *        + (lambda u / 2) K13 ((s_f.k)(s_i.beta) + (s_f.beta)(s_i.k))      (Eq. F2)
 *   F3 = K23 + (u (s_i.beta) + lambda (s_f.beta)) K13
 *        - (lambda u / 2) IntK13 ((s_f.eps)(s_i.eps) - (s_f.beta)(s_i.beta))
 *        + (kappa/2) K23 (s_f.s_i) - (lambda u / 2) K23 (s_f.k)(s_i.k)       (Eq. F3)
 * with kappa~ = 1/(1-lambda) - (1-lambda). */
void orc_nlc_stokes(double lam, const double bes[3], const double si[3], const double sf[3],
                    const double eps[3], const double beta[3], const double k[3], double F[4])
{
    double one_m = 1.0 - lam;
    double u = lam / one_m;
    double kappa = 1.0 / one_m + one_m;
    double kappat = 1.0 / one_m - one_m;
    double K13 = bes[0], K23 = bes[1], IK = bes[2];
    double w, g[3];
    orc_nlc_wg(lam, bes, si, eps, beta, k, &w, g);
    double sie = dot3(si, eps), sib = dot3(si, beta), sik = dot3(si, k);
    double sfe = dot3(sf, eps), sfb = dot3(sf, beta), sfk = dot3(sf, k);
    double fxi[3];
    cross3(sf, si, fxi);
    double lu2 = lam * u / 2.0;
    F[0] = w + dot3(sf, g);
    F[1] = -K13 * (u * sie + lam * sfe) - lu2 * IK * (sfe * sib + sfb * sie) + (kappat / 2.0) * K23 * dot3(fxi, k);
    F[2] = (kappat / 2.0) * K13 * dot3(fxi, eps) - (lam * IK - kappat * K23) * sik - (u * IK - kappat * K23) * sfk +
           lu2 * K13 * (sfk * sib + sfb * sik);
    F[3] = K23 + (u * sib + lam * sfb) * K13 - lu2 * IK * (sfe * sie - sfb * sib) + (kappa / 2.0) * K23 * dot3(sf, si) -
           lu2 * K23 * sfk * sik;
}

/* NBW, App. A.2 / Sec. 3.1.  lambda = positron momentum fraction.
 *   w0  = IntK13(u~') + rho K23 - xi3 K23                                   (Eq. w0)
 *   j_e = (1/(1-l) - xi3/l) K13 beta + xi1 (1/l) K13 eps
 *         + xi2 ((1/(1-l)) IntK13 + rho~ K23) k                              (Eq. j_e)
 *   j_p = (-1/l + xi3/(1-l)) K13 beta - xi1 (1/(1-l)) K13 eps
 *         + xi2 ((1/l) IntK13 - rho~ K23) k                                  (Eq. j_p)
 * rho = (1-l)/l + l/(1-l), rho~ = (1-l)/l - l/(1-l), u~' = 2 (1/l + 1/(1-l)) / (3 chi). */
void orc_nbw_j(double lam, const double bes[3], const double xi[3], const double eps[3], const double beta[3],
               const double k[3], double *w0, double je[3], double jp[3])
{
    double one_m = 1.0 - lam;
    double rho = one_m / lam + lam / one_m;
    double rhot = one_m / lam - lam / one_m;
    double K13 = bes[0], K23 = bes[1], IK = bes[2];
    *w0 = IK + rho * K23 - xi[2] * K23;
    double eb = (1.0 / one_m - xi[2] / lam) * K13, ee = xi[0] * (1.0 / lam) * K13,
           ek = xi[1] * ((1.0 / one_m) * IK + rhot * K23);
    double pb = (-1.0 / lam + xi[2] / one_m) * K13, pe = -xi[0] * (1.0 / one_m) * K13,
           pk = xi[1] * ((1.0 / lam) * IK - rhot * K23);
    for (int i = 0; i < 3; ++i) {
        je[i] = eb * beta[i] + ee * eps[i] + ek * k[i];
        jp[i] = pb * beta[i] + pe * eps[i] + pk * k[i];
    }
}

/* NBW full spectrum G = G0 + xi1 G1 + xi2 G2 + xi3 G3 (Eqs. G0-G3 of App. A.2).
 * The last term of G3 takes the sign of its Airy form, +(1 - rho/2) K23 (s_p.k)(s_e.k);
 * the printed Bessel form has the opposite sign (reading recorded in the design notes). */
void orc_nbw_G(double lam, const double bes[3], const double sp[3], const double se[3], const double eps[3],
               const double beta[3], const double k[3], double G[4])
{
    double one_m = 1.0 - lam;
    double rho = one_m / lam + lam / one_m;
    double rhot = one_m / lam - lam / one_m;
    double ut = 1.0 / lam + 1.0 / one_m;
    double K13 = bes[0], K23 = bes[1], IK = bes[2];
    double spe = dot3(sp, eps), spb = dot3(sp, beta), spk = dot3(sp, k);
    double see = dot3(se, eps), seb = dot3(se, beta), sek = dot3(se, k);
    double pxe[3];
    cross3(sp, se, pxe);
    G[0] = IK + rho * K23 + (1.0 / one_m) * seb * K13 - (1.0 / lam) * spb * K13 + (IK - 2.0 * K23) * dot3(sp, se) +
           (rho * IK - (rho - 2.0) * K23) * spk * sek;
    G[1] = K13 * ((1.0 / lam) * see - (1.0 / one_m) * spe) - (ut / 2.0) * IK * (spe * seb + spb * see) +
           (rhot / 2.0) * K23 * dot3(pxe, k);
    G[2] = -(ut / 2.0) * K13 * dot3(pxe, eps) + ((1.0 / one_m) * IK + rhot * K23) * sek +
           ((1.0 / lam) * IK - rhot * K23) * spk - (rhot / 2.0) * K13 * (spk * seb + spb * sek);
    G[3] = -K23 + (-(1.0 / lam) * seb + (1.0 / one_m) * spb) * K13 - (ut / 2.0) * IK * (spe * see - spb * seb) +
           (rho / 2.0) * K23 * dot3(sp, se) + (1.0 - rho / 2.0) * K23 * spk * sek;
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n (textbook).       */
/* ------------------------------------------------------------------------- */
#define ORC_GL_MAX 64
static int gl_n = 10;                 /* Gauss-Legendre points per panel */
static double panel_w = 1.0 / 16.0;  /* panel width in the substituted variable t */
static double gl_x[ORC_GL_MAX], gl_w[ORC_GL_MAX];
static int gl_ready = 0;

/* Select the quadrature rule used by every integral below (tests use this to
 * show that the default rule has converged). */
int orc_set_quadrature(int n_points, double width)
{
    if (n_points < 2 || n_points > ORC_GL_MAX || !(width > 0.0)) return -1;
    gl_n = n_points;
    panel_w = width;
    gl_ready = 0;
    return 0;
}

static void gl_init(void)
{
    if (gl_ready) return;
    int n = gl_n;
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    gl_ready = 1;
}

/* ------------------------------------------------------------------------- */
/* Integrands of the rates in the substituted variables.                       */
/* NLC: variable t with u' = t^3 (removes the lambda^{-2/3} infrared behaviour, */
/*      Sec. 4.2), lambda = 3 chi u' / (2 + 3 chi u'), d lambda/du' = 6 chi /   */
/*      (2 + 3 chi u')^2.  Integrand = w_sigma(lambda) d lambda/dt.             */
/* NBW: folded positron spectrum (symmetric in lambda <-> 1-lambda); variable   */
/*      t with u~' = u~'_min + t^2, u~'_min = 8/(3 chi); the density in t of     */
/*      one half is w0(u~') * 4 / (3 chi u~'^{3/2}); scaled by e^{u~'_min}.     */
/* sigma: +1 (up / xi3=+1), -1 (down / xi3=-1), 0 (average).                   */
/* ------------------------------------------------------------------------- */
static double nlc_integrand_t(double chi, int sigma, double t)
{
    if (t <= 0.0) {
        /* limit t -> 0: w ~ 2 K23(t^3) ~ 2 * 2^{-1/3} Gamma(2/3) t^{-2}; times 3 t^2 * 6 chi / 4 */
        double g23 = 1.35411793942640041695; /* Gamma(2/3) */
        return 2.0 * 0.5 * g23 * pow(2.0, 2.0 / 3.0) * 3.0 * 6.0 * chi / 4.0;
    }
    double up = t * t * t;
    double den = 2.0 + 3.0 * chi * up;
    double lam = 3.0 * chi * up / den;
    double one_m = 2.0 / den;
    double bes[3];
    orc_bessel(up, bes);
    double kappa = 1.0 / one_m + one_m;
    double w = -bes[2] + kappa * bes[1] + lam * (double)sigma * bes[0];
    return w * 6.0 * chi / (den * den) * 3.0 * t * t;
}

static double nbw_integrand_t(double chi, int sigma, double t)
{
    double umin = 8.0 / (3.0 * chi);
    double ut = umin + t * t;
    double rho = 1.5 * chi * ut - 2.0; /* rho = 1/(l(1-l)) - 2 with l(1-l) = 2/(3 chi u~') */
    double bes[3];
    orc_bessel_scaled(ut, bes);
    double w0 = bes[2] + rho * bes[1] - (double)sigma * bes[1];
    return w0 * exp(-t * t) * 4.0 / (3.0 * chi * ut * sqrt(ut));
}

static double integrand_t(int nbw, double chi, int sigma, double t)
{
    return nbw ? nbw_integrand_t(chi, sigma, t) : nlc_integrand_t(chi, sigma, t);
}

static double gl_segment(int nbw, double chi, int sigma, double a, double b)
{
    gl_init();
    double m = 0.5 * (a + b), r = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < gl_n; ++i) s += gl_w[i] * integrand_t(nbw, chi, sigma, m + r * gl_x[i]);
    return s * r;
}

/* Panel layout in t: NLC t in [0, 80^{1/3}], NBW t in [0, sqrt(80)], panels of width panel_w. */
#define ORC_PANEL_W panel_w
static double t_end(int nbw) { return nbw ? sqrt(80.0) : cbrt(80.0); }

/* Rate integrals (Sec. 5.1 rate tabulation, App. A):
 *   NLC: I_sigma(chi) = int_0^1 [-IntK13(u') + kappa K23(u') + sigma lambda K13(u')] d lambda,
 *        W_sigma = alpha/(sqrt3 pi eta0 gamma) * I_sigma  (per unit time 1/omega).
 *   NBW: J_sigma(chi) = int_0^1 [IntK13(u~') + rho K23(u~') - sigma K23(u~')] d lambda,
 *        W_sigma = alpha/(sqrt3 pi eta0 eps_gamma) * J_sigma; returned scaled by e^{8/(3 chi)}. */
double orc_rate_integral(int nbw, double chi, int sigma)
{
    double T = t_end(nbw), s = 0.0;
    int np = (int)ceil(T / ORC_PANEL_W);
    for (int p = 0; p < np; ++p) {
        double a = p * ORC_PANEL_W, b = fmin(T, (p + 1) * ORC_PANEL_W);
        s += gl_segment(nbw, chi, sigma, a, b);
    }
    return nbw ? 2.0 * s : s;
}

/* Normalised cumulative distribution of the sampled variable at t (NLC: from
 * lambda = 0; NBW: folded, from the centre lambda = 1/2 outwards). */
double orc_cdf_t(int nbw, double chi, int sigma, double t)
{
    double T = t_end(nbw), total = 0.0, part = 0.0;
    int np = (int)ceil(T / ORC_PANEL_W);
    for (int p = 0; p < np; ++p) {
        double a = p * ORC_PANEL_W, b = fmin(T, (p + 1) * ORC_PANEL_W);
        double seg = gl_segment(nbw, chi, sigma, a, b);
        total += seg;
        if (b <= t) part += seg;
        else if (a < t) part += gl_segment(nbw, chi, sigma, a, t);
    }
    return part / total;
}

/* ------------------------------------------------------------------------- */
/* Tables (Sec. 5.1: rates W_up/W_down and ICDFs IntF^-1_up/down; Sec. 5.2:    */
/* W_+/W_- and IntG^-1_+/-).                                                    */
/*   chi grid:  chi_i = exp(ln chi_min + i * dlnchi), i < n_chi                 */
/*   r grid:    y_m = y_lo + m * dy (logit of the cumulative probability r)     */
/*   rate:      NLC ln I_sigma(chi_i);  NBW ln(J_sigma(chi_i) e^{8/(3 chi_i)})   */
/*   ICDF:      NLC ln u'(chi_i, r_m);  NBW ln x(chi_i, r_m), x = u~' - 8/(3chi) */
/* sigma index 0 = up / xi3=+1 (sigma=+1), index 1 = down / xi3=-1 (sigma=-1). */
/* ------------------------------------------------------------------------- */
typedef struct {
    double chi_min, chi_max;
    int32_t n_chi, n_r;
    double y_lo, y_hi;
} orc_table_desc;

typedef struct {
    orc_table_desc d;
    double *nlc_rate; /* [2][n_chi] */
    double *nbw_rate; /* [2][n_chi] */
    double *nlc_icdf; /* [2][n_chi][n_r] */
    double *nbw_icdf; /* [2][n_chi][n_r] */
    double *amm;      /* [n_chi] ln a(chi_i), the field-dependent anomalous moment; NULL if not built */
} orc_tables;

/* Solve c(t) = r for t by bisection on the panel that brackets r, followed by
 * Newton steps (derivative = integrand) kept inside the bracket. */
static double invert_row(int nbw, double chi, int sigma, const double *cum, int np, double total, double r)
{
    double target = r * total;
    int p = 0;
    while (p < np - 1 && cum[p + 1] < target) ++p;
    double T = t_end(nbw);
    double a = p * ORC_PANEL_W, b = fmin(T, (p + 1) * ORC_PANEL_W);
    double base = cum[p];
    double lo = a, hi = b;
    double t = a + (b - a) * (target - base) / (cum[p + 1] - base);
    for (int it = 0; it < 200; ++it) {
        double f = base + gl_segment(nbw, chi, sigma, a, t) - target;
        if (f > 0) hi = t; else lo = t;
        double d = integrand_t(nbw, chi, sigma, t);
        double tn = t - f / d;
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (fabs(tn - t) <= 1e-15 * fmax(t, 1e-300) || hi - lo <= 1e-15 * hi) { t = tn; break; }
        t = tn;
    }
    return t;
}

static void build_row(int nbw, const orc_table_desc *d, double chi, int sigma, double *rate_out, double *icdf_out)
{
    double T = t_end(nbw);
    int np = (int)ceil(T / ORC_PANEL_W);
    double *cum = (double *)malloc(sizeof(double) * (np + 1));
    cum[0] = 0.0;
    for (int p = 0; p < np; ++p) {
        double a = p * ORC_PANEL_W, b = fmin(T, (p + 1) * ORC_PANEL_W);
        cum[p + 1] = cum[p] + gl_segment(nbw, chi, sigma, a, b);
    }
    double total = cum[np];
    *rate_out = nbw ? log(2.0 * total) : log(total);
    double dy = (d->y_hi - d->y_lo) / (d->n_r - 1);
    for (int m = 0; m < d->n_r; ++m) {
        double y = d->y_lo + m * dy;
        double r = 1.0 / (1.0 + exp(-y));
        double t = invert_row(nbw, chi, sigma, cum, np, total, r);
        /* NLC stores ln u' = 3 ln t; NBW stores ln x = 2 ln t */
        icdf_out[m] = nbw ? 2.0 * log(t) : 3.0 * log(t);
    }
    free(cum);
}

int orc_tables_build(const orc_table_desc *d, double *nlc_rate, double *nbw_rate, double *nlc_icdf, double *nbw_icdf)
{
    if (d->n_chi < 2 || d->n_r < 4 || !(d->chi_min > 0) || !(d->chi_max > d->chi_min) || !(d->y_hi > d->y_lo)) return -1;
    gl_init();
    double dl = (log(d->chi_max) - log(d->chi_min)) / (d->n_chi - 1);
    int total = 4 * d->n_chi;
#pragma omp parallel for schedule(dynamic, 1)
    for (int job = 0; job < total; ++job) {
        int nbw = job / (2 * d->n_chi);
        int s = (job / d->n_chi) % 2;
        int i = job % d->n_chi;
        double chi = exp(log(d->chi_min) + i * dl);
        int sigma = s == 0 ? +1 : -1;
        double *rate = (nbw ? nbw_rate : nlc_rate) + s * d->n_chi + i;
        double *icdf = (nbw ? nbw_icdf : nlc_icdf) + ((size_t)s * d->n_chi + i) * d->n_r;
        build_row(nbw, d, chi, sigma, rate, icdf);
    }
    return 0;
}

/* ---- table lookups (the interpolation rules are part of the table's definition) ---- */

/* chi row coordinate: s = (ln chi - ln chi_min) / dlnchi -> (i, f), clamped to the grid. */
static void chi_coord(const orc_table_desc *d, double chi, int *i, double *f)
{
    double dl = (log(d->chi_max) - log(d->chi_min)) / (d->n_chi - 1);
    double s = (log(chi) - log(d->chi_min)) / dl;
    if (s <= 0.0) { *i = 0; *f = 0.0; return; }
    if (s >= d->n_chi - 1) { *i = d->n_chi - 2; *f = 1.0; return; }
    int ii = (int)floor(s);
    if (ii > d->n_chi - 2) ii = d->n_chi - 2;
    *i = ii;
    *f = s - ii;
}

/* NLC rate integral I_sigma(chi): linear in (ln chi, ln I) inside the grid;
 * below chi_min proportional to chi (classical limit); above chi_max clamped. */
double orc_nlc_rate_lookup(const orc_tables *t, int s, double chi, int *clamped)
{
    const orc_table_desc *d = &t->d;
    const double *L = t->nlc_rate + s * d->n_chi;
    if (clamped) *clamped = chi > d->chi_max;
    if (chi < d->chi_min) return exp(L[0]) * (chi / d->chi_min);
    int i; double f;
    chi_coord(d, chi, &i, &f);
    return exp((1.0 - f) * L[i] + f * L[i + 1]);
}

/* NBW rate integral J_sigma(chi): linear in (ln chi, ln(J e^{8/(3chi)})); zero below chi_min. */
double orc_nbw_rate_lookup(const orc_tables *t, int s, double chi, int *clamped)
{
    const orc_table_desc *d = &t->d;
    const double *L = t->nbw_rate + s * d->n_chi;
    if (clamped) *clamped = chi > d->chi_max;
    if (chi < d->chi_min) return 0.0;
    int i; double f;
    chi_coord(d, chi, &i, &f);
    double chic = chi > d->chi_max ? d->chi_max : chi;
    return exp((1.0 - f) * L[i] + f * L[i + 1] - 8.0 / (3.0 * chic));
}

/* One ICDF row at logit coordinate y: cubic (4-point Lagrange) in y inside the
 * grid; below y_lo the asymptote (NLC: u' ~ r^3, NBW: x ~ r^2 -> slope 3 or 2
 * in y); above y_hi the last value. */
static double icdf_row(const double *row, const orc_table_desc *d, int nbw, double y)
{
    double dy = (d->y_hi - d->y_lo) / (d->n_r - 1);
    double tt = (y - d->y_lo) / dy;
    if (tt <= 0.0) return row[0] + (nbw ? 2.0 : 3.0) * (y - d->y_lo);
    if (tt >= d->n_r - 1) return row[d->n_r - 1];
    int m = (int)floor(tt);
    if (m < 1) m = 1;
    if (m > d->n_r - 3) m = d->n_r - 3;
    double x = tt - m;
    double wm1 = -x * (x - 1.0) * (x - 2.0) / 6.0;
    double w0 = (x + 1.0) * (x - 1.0) * (x - 2.0) / 2.0;
    double w1 = -(x + 1.0) * x * (x - 2.0) / 2.0;
    double w2 = (x + 1.0) * x * (x - 1.0) / 6.0;
    return wm1 * row[m - 1] + w0 * row[m] + w1 * row[m + 1] + w2 * row[m + 2];
}

/* ICDF lookup: ln of the sampled variable (NLC: u'; NBW: x) for chi and the
 * uniform r; rows of the two bracketing chi nodes blended linearly in ln chi. */
double orc_icdf_lookup(const orc_tables *t, int nbw, int s, double chi, double r)
{
    const orc_table_desc *d = &t->d;
    const double *base = (nbw ? t->nbw_icdf : t->nlc_icdf) + (size_t)s * d->n_chi * d->n_r;
    int i; double f;
    chi_coord(d, chi, &i, &f);
    double y = log(r) - log(1.0 - r);
    double v0 = icdf_row(base + (size_t)i * d->n_r, d, nbw, y);
    double v1 = icdf_row(base + (size_t)(i + 1) * d->n_r, d, nbw, y);
    return (1.0 - f) * v0 + f * v1;
}

/* NLC: lambda from u' (Sec. 5.1 definitions u = lambda/(1-lambda), u' = 2u/(3chi)). */
double orc_nlc_lambda(double chi, double up) { return 3.0 * chi * up / (2.0 + 3.0 * chi * up); }

/* NBW: positron fraction from the folded variable x and the uniform r
 * (r < 1/2 -> lambda < 1/2 side, r >= 1/2 -> lambda >= 1/2 side). */
double orc_nbw_mu(double chi, double x)
{
    double umin = 8.0 / (3.0 * chi);
    double ut = umin + x;
    /* mu (1 - mu) = 2 / (3 chi u~'),  mu <= 1/2 */
    double q = 2.0 / (3.0 * chi * ut);
    return 0.5 * (1.0 - sqrt(1.0 - 4.0 * q));
}

/* ------------------------------------------------------------------------- */
/* One-loop self-energy terms (App. A.1) and the field-dependent anomalous     */
/* moment g(chi) = 2 + 2 a(chi) (Sec. 8.6.2).                                  */
/*                                                                            */
/* Airy and Scorer functions from their integral definition (App. A.1):       */
/*   Ai(z) + i Gi(z) = (1/pi) int_0^inf exp(i (z t + t^3/3)) dt.               */
/* For z >= 0 the integrand is analytic and bounded in the sector             */
/* 0 <= arg t <= pi/6 (there Re(i t^3) <= 0 and Re(i z t) <= 0), so by Cauchy  */
/* the ray t = e^{i pi/6} s gives the same integral, now absolutely convergent:*/
/*   Ai + i Gi = (e^{i pi/6}/pi) int_0^inf exp(-s^3/3 - z s/2)                 */
/*                                   exp(i sqrt(3) z s / 2) ds.               */
/* Gauss-Legendre panels on [0, S], S where the exponent reaches -45.  Gi has  */
/* no cancellation (Gi ~ 1/(pi z) for large z); Ai does (it decays like        */
/* exp(-2 z^{3/2}/3) from terms of size 1/z), so Ai is accurate to ~1e-16 in   */
/* absolute terms only.                                                       */
/* ------------------------------------------------------------------------- */
void orc_airy_scorer(double z, double out[2])
{
    gl_init();
    double S = fmin(cbrt(135.0), 90.0 / fmax(z, 1e-300));
    const int np = 48;
    double h = S / np, c = 0.0, sn = 0.0;
    double w = 0.5 * ORC_SQRT3 * z;
    for (int p = 0; p < np; ++p) {
        double a = p * h, r = 0.5 * h;
        for (int k = 0; k < gl_n; ++k) {
            double s = a + r + r * gl_x[k];
            double e = exp(-s * s * s / 3.0 - 0.5 * z * s) * gl_w[k] * r;
            c += e * cos(w * s);
            sn += e * sin(w * s);
        }
    }
    /* e^{i pi/6} = (sqrt(3)/2, 1/2) */
    out[0] = (0.5 * ORC_SQRT3 * c - 0.5 * sn) / ORC_PI; /* Ai */
    out[1] = (0.5 * c + 0.5 * ORC_SQRT3 * sn) / ORC_PI; /* Gi */
}

/* Field-dependent anomalous moment from the Scorer term of the loop (App. A.1, the Gi(z)/sqrt(z) part of
 * R_if), with z = (u/chi)^{2/3}, u = lambda/(1 - lambda):
 *   a(chi) = (alpha/chi) int_0^1 dlambda lambda Gi(z)/sqrt(z)
 *          = (alpha/chi) int_0^inf du u/(1+u)^3 Gi(z)/sqrt(z).
 * Normalised so that chi -> 0 gives Schwinger's alpha/(2 pi) (Gi(z) -> 1/(pi z)).  With u = chi v^3
 * (z = v^2) and v = e^t:  a(chi) = 3 alpha chi int v^5 Gi(v^2)/(1 + chi v^3)^3 dt, a smooth integrand on
 * t in [ln(1e-3 m), ln(1e3 M)], m = min(1, chi^{-1/3}), M = max(1, chi^{-1/3}) (the ends contribute below
 * 1e-15 of the result); Gauss-Legendre panels of width 1/8 in t. */
double orc_amm(double chi)
{
    gl_init();
    double c3 = cbrt(1.0 / chi);
    double t0 = log(1e-3 * fmin(1.0, c3)), t1 = log(1e3 * fmax(1.0, c3));
    int np = (int)ceil((t1 - t0) * 8.0);
    double h = (t1 - t0) / np, acc = 0.0;
    for (int p = 0; p < np; ++p) {
        double a = t0 + p * h, r = 0.5 * h;
        for (int k = 0; k < gl_n; ++k) {
            double t = a + r + r * gl_x[k];
            double v = exp(t);
            double ag[2];
            orc_airy_scorer(v * v, ag);
            double d = 1.0 + chi * v * v * v;
            acc += gl_w[k] * r * pow(v, 5.0) * ag[1] / (d * d * d);
        }
    }
    return 3.0 * ORC_ALPHA * chi * acc;
}

/* Table of ln a(chi_i) on the rate grid (one entry per chi node). */
int orc_amm_build(const orc_table_desc *d, double *amm)
{
    if (d->n_chi < 2 || !(d->chi_min > 0) || !(d->chi_max > d->chi_min)) return -1;
    gl_init();
    double dl = (log(d->chi_max) - log(d->chi_min)) / (d->n_chi - 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < d->n_chi; ++i) amm[i] = log(orc_amm(exp(log(d->chi_min) + i * dl)));
    return 0;
}

/* a(chi) from the table: linear in (ln chi, ln a) between nodes, the end values outside the grid
 * (below chi_min a(chi) differs from alpha/(2 pi) by less than 1e-6 of it).  Returns the zero-field value
 * alpha/(2 pi) if no table was built. */
double orc_amm_lookup(const orc_tables *t, double chi)
{
    if (!t->amm) return ORC_ALPHA / (2.0 * ORC_PI);
    int i; double f;
    chi_coord(&t->d, chi > 0.0 ? chi : t->d.chi_min, &i, &f);
    return exp((1.0 - f) * t->amm[i] + f * t->amm[i + 1]);
}

/* ------------------------------------------------------------------------- */
/* Fields: analytic plane waves propagating along z (stand-in for the PIC      */
/* grid fields of Sec. 4).  E, B in units of m c omega / e.                     */
/* ------------------------------------------------------------------------- */
enum { ORC_FIELD_CONST = 0, ORC_FIELD_LP = 1, ORC_FIELD_CP = 2, ORC_FIELD_CP_COUNTER = 3, ORC_FIELD_ROT_B = 4 };
typedef struct {
    int32_t kind;
    int32_t pad;
    double a0, n_cycles, phase; /* phi = t - z + phase (second pulse: t + z + phase) */
    double E0[3], B0[3];        /* constant fields (kind CONST) */
    double eta0;                /* hbar omega / m c^2 */
} orc_field;

static double envelope(double phi, double n)
{
    if (phi < 0.0 || phi > 2.0 * ORC_PI * n) return 0.0;
    double s = sin(phi / (2.0 * n));
    return s * s;
}

void orc_field_eval(const orc_field *f, const double x[3], double t, double E[3], double B[3])
{
    for (int i = 0; i < 3; ++i) { E[i] = 0.0; B[i] = 0.0; }
    if (f->kind == ORC_FIELD_CONST) {
        for (int i = 0; i < 3; ++i) { E[i] = f->E0[i]; B[i] = f->B0[i]; }
        return;
    }
    if (f->kind == ORC_FIELD_ROT_B) {
        /* a magnetic field of constant strength |B0_z| that turns from z to y (the rotating-field test of
         * Sec. 8.3): angle (pi/2) clamp((t + phase) / (2 pi n_cycles), 0, 1), uniform in space, E = 0 */
        double u = (t + f->phase) / (2.0 * ORC_PI * f->n_cycles);
        u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
        double th = 0.5 * ORC_PI * u;
        B[1] = f->B0[2] * sin(th);
        B[2] = f->B0[2] * cos(th);
        return;
    }
    double phi = t - x[2] + f->phase;
    double a = f->a0 * envelope(phi, f->n_cycles);
    double ex = a * cos(phi), ey = f->kind == ORC_FIELD_LP ? 0.0 : a * sin(phi);
    /* forward wave: B = z x E */
    E[0] = ex; E[1] = ey;
    B[0] = -ey; B[1] = ex;
    if (f->kind == ORC_FIELD_CP_COUNTER) {
        double phi2 = t + x[2] + f->phase;
        double a2 = f->a0 * envelope(phi2, f->n_cycles);
        double ex2 = a2 * cos(phi2), ey2 = a2 * sin(phi2);
        /* backward wave: B = -z x E */
        E[0] += ex2; E[1] += ey2;
        B[0] += ey2; B[1] += -ex2;
    }
}

/* Fields at n points (x: [n][3]; E, B: [n][3]), for tests and diagnostics. */
void orc_field_eval_n(const orc_field *f, int64_t n, const double *x, double t, double *E, double *B)
{
    for (int64_t i = 0; i < n; ++i) orc_field_eval(f, x + 3 * i, t, E + 3 * i, B + 3 * i);
}

/* ------------------------------------------------------------------------- */
/* Particles (structure of arrays, FP64) and step parameters                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    double *x, *y, *z, *px, *py, *pz, *sx, *sy, *sz, *tau, *w;
    uint64_t *id;
    int64_t n, capacity;
} orc_particles;

enum {
    ORC_F_TAU = 1u << 0,           /* optical-depth decision (else per-step probability r1 < W dt) */
    ORC_F_RECOIL = 1u << 1,        /* radiation reaction: p <- (1 - lambda) p */
    ORC_F_SPIN_COLLAPSE = 1u << 2, /* s_f = +-S_SQA (else s_f = <s_f> = g/w) */
    ORC_F_POL_COLLAPSE = 1u << 3,  /* xi = +-Xi_PQA (else xi = F/F0) */
    ORC_F_NONTRANSITION = 1u << 4, /* spin / polarization update when nothing happens (Sec. 6) */
    ORC_F_PUSH = 1u << 5,          /* Boris momentum push */
    ORC_F_TBMT = 1u << 6,          /* T-BMT spin precession */
    ORC_F_TBMT_PAPER = 1u << 7,    /* T-BMT coefficient as printed in Sec. 8.3 */
    ORC_F_EMIT = 1u << 8,          /* QED events (NLC for leptons, NBW for photons) */
    ORC_F_RESOLVED = 1u << 9,      /* rates and sampling depend on s.beta (leptons) / xi3 (photons) */
    ORC_F_MOVE = 1u << 10,         /* position advance */
    ORC_F_SPIN_EVENT = 1u << 11,   /* lepton spin changes at emission; pair daughters get spins */
    ORC_F_POL_EVENT = 1u << 12,    /* emitted photons get the Stokes vector of F (else unpolarized) */
    ORC_F_AMM = 1u << 13,          /* T-BMT with the field-dependent a(chi) (Sec. 8.6.2) instead of alpha/(2 pi) */
    ORC_F_LOOP = 1u << 14,         /* Scorer term of the loop in the no-emission update; T-BMT with g = 2 */
    ORC_F_G2 = 1u << 15,           /* T-BMT with g = 2 (a = 0), the comparison run of Sec. 8.6.2 */
    ORC_F_BETA_BASIS = 1u << 16,   /* spins resolved along +-beta instead of the SQA (Sec. 8.3 comparison) */
    ORC_F_REJECT = 1u << 17,       /* table-free decision and sampling by rejection (Sec. 4.2) */
    ORC_F_MIX_QUANTILE = 1u << 18  /* emission's u' the exact quantile of the spin mixture at r2 (oracle only) */
};

void orc_mlp_target(double chi, double r, double s, double out[4]); /* defined with the sampler's target */

typedef struct {
    double dt, t;         /* step length, time at the start of the step */
    uint64_t step, seed;
    uint32_t flags;
    uint32_t pad;
    double photon_store_min; /* photons with |k| below this are not stored */
    double chi_floor;        /* no QED below this chi */
} orc_step;

typedef struct {
    int64_t events, stored, dropped_capacity, chi_clamped, renormalised, below_store;
    int64_t bound_exceeded; /* rejection steps whose acceptance probability exceeded 1 */
} orc_counters;

/* result record of one particle's step, appended serially afterwards */
typedef struct {
    int event, store;
    double d0[3], k0[3], P0[3], tau0, w0;      /* daughter 0 (photon / electron) */
    double d1k[3], s1[3], tau1;                /* daughter 1 (positron) */
    uint64_t id0, id1;
    int clamped, renorm, bound;
    double kept_p[3], kept_s[3], kept_tau;     /* lepton state if its event is not applied */
} orc_result;

static void push_particle(orc_particles *b, const double x[3], const double p[3], const double s[3], double tau,
                          double w, uint64_t id)
{
    int64_t j = b->n++;
    b->x[j] = x[0]; b->y[j] = x[1]; b->z[j] = x[2];
    b->px[j] = p[0]; b->py[j] = p[1]; b->pz[j] = p[2];
    b->sx[j] = s[0]; b->sy[j] = s[1]; b->sz[j] = s[2];
    b->tau[j] = tau; b->w[j] = w; b->id[j] = id;
}

/* Photon polarization vector P from Stokes xi in the basis (eps, beta, k),
 * Sec. 3.2: P = xi2 k + l (cos(dth) eps + sin(dth) beta), l = sqrt(xi1^2 + xi3^2),
 * 2 dth = atan2(xi1, xi3) (the paper's unit-vector form, generalised to |xi| <= 1). */
void orc_stokes_to_P(const double xi[3], const double eps[3], const double beta[3], const double k[3], double P[3])
{
    double l = sqrt(xi[0] * xi[0] + xi[2] * xi[2]);
    double dth = 0.5 * atan2(xi[0], xi[2]);
    double c = l * cos(dth), s = l * sin(dth);
    for (int i = 0; i < 3; ++i) P[i] = xi[1] * k[i] + c * eps[i] + s * beta[i];
}

/* Stokes from P in the basis (eps, beta, k), Sec. 3.2 Eq. (P-vector/Stokes relation):
 * xi1 = 2 P1 P2 / l, xi2 = P.k, xi3 = (P1^2 - P2^2)/l, l = sqrt(P1^2 + P2^2). */
void orc_P_to_stokes(const double P[3], const double eps[3], const double beta[3], const double k[3], double xi[3])
{
    double P1 = dot3(P, eps), P2 = dot3(P, beta);
    double l = sqrt(P1 * P1 + P2 * P2);
    xi[1] = dot3(P, k);
    if (l > 0.0) {
        xi[0] = 2.0 * P1 * P2 / l;
        xi[2] = (P1 * P1 - P2 * P2) / l;
    } else {
        xi[0] = 0.0;
        xi[2] = 0.0;
    }
}

/* Local basis (Sec. 3): k = direction of motion; eps along the component of the
 * Lorentz-force field f perpendicular to k; beta = k x eps (right-handed).
 * Leptons: f = E + v x B, eps = -q f_perp/|f_perp| (q = charge); photons: f = E + k x B, eps = f_perp/|f_perp|.
 * Returns 0 if the basis is undefined. */
static int make_basis(const double E[3], const double B[3], const double v[3], const double khat[3], double sign,
                      double eps[3], double beta[3])
{
    double vxB[3];
    cross3(v, B, vxB);
    double f[3] = {E[0] + vxB[0], E[1] + vxB[1], E[2] + vxB[2]};
    double fk = dot3(f, khat);
    double fp[3] = {f[0] - fk * khat[0], f[1] - fk * khat[1], f[2] - fk * khat[2]};
    double n = sqrt(dot3(fp, fp));
    if (!(n > 0.0)) return 0;
    for (int i = 0; i < 3; ++i) eps[i] = sign * fp[i] / n;
    cross3(khat, eps, beta);
    return 1;
}

/* chi of a particle with momentum p (energy e) in E, B (standard invariant,
 * chi = eta0 sqrt((e E + p x B)^2 - (p . E)^2); Sec. 1, Eq. for chi_e). */
static double chi_of(double eta0, double e, const double p[3], const double E[3], const double B[3])
{
    double pxB[3];
    cross3(p, B, pxB);
    double a[3] = {e * E[0] + pxB[0], e * E[1] + pxB[1], e * E[2] + pxB[2]};
    double pe = dot3(p, E);
    double v = dot3(a, a) - pe * pe;
    return eta0 * sqrt(v > 0.0 ? v : 0.0);
}

/* chi_of for tests */
double orc_chi(double eta0, double e, const double p[3], const double E[3], const double B[3])
{
    return chi_of(eta0, e, p, E, B);
}

/* Rodrigues rotation of s about the unit axis n by angle th. */
static void rotate(double s[3], const double n[3], double th)
{
    double c = cos(th), sn = sin(th);
    double nxs[3];
    cross3(n, s, nxs);
    double ns = dot3(n, s);
    for (int i = 0; i < 3; ++i) s[i] = s[i] * c + nxs[i] * sn + n[i] * ns * (1.0 - c);
}

/* ------------------------------------------------------------------------- */
/* Lepton step: Boris push, T-BMT precession, position advance, then the NLC  */
/* module (Sec. 5.1 and its flow chart; non-emission update Sec. 6).           */
/* ------------------------------------------------------------------------- */
static void lepton_one(const orc_tables *tb, const orc_field *fd, const orc_step *st, int q, orc_particles *L,
                       int64_t j, orc_result *res)
{
    const uint32_t fl = st->flags;
    const double dt = st->dt;
    const double aE = ORC_ALPHA / (2.0 * ORC_PI); /* anomalous moment a_e = alpha/(2 pi) */
    memset(res, 0, sizeof(*res));
    double x[3] = {L->x[j], L->y[j], L->z[j]};
    double p[3] = {L->px[j], L->py[j], L->pz[j]};
    double s[3] = {L->sx[j], L->sy[j], L->sz[j]};
    double tau = L->tau[j];
    uint64_t id = L->id[j];
    double E[3], B[3];
    orc_field_eval(fd, x, st->t, E, B);

    /* Boris push (Sec. 5.1 "classical Lorentz pusher") */
    double pold[3] = {p[0], p[1], p[2]};
    if (fl & ORC_F_PUSH) {
        double h = 0.5 * q * dt;
        double pm[3] = {p[0] + h * E[0], p[1] + h * E[1], p[2] + h * E[2]};
        double gm = sqrt(1.0 + dot3(pm, pm));
        double tv[3] = {h * B[0] / gm, h * B[1] / gm, h * B[2] / gm};
        double t2 = dot3(tv, tv);
        double sv[3] = {2.0 * tv[0] / (1.0 + t2), 2.0 * tv[1] / (1.0 + t2), 2.0 * tv[2] / (1.0 + t2)};
        double c1[3];
        cross3(pm, tv, c1);
        double pp[3] = {pm[0] + c1[0], pm[1] + c1[1], pm[2] + c1[2]};
        double c2[3];
        cross3(pp, sv, c2);
        double pl[3] = {pm[0] + c2[0], pm[1] + c2[1], pm[2] + c2[2]};
        for (int i = 0; i < 3; ++i) p[i] = pl[i] + h * E[i];
    }

    /* T-BMT precession (Sec. 8.3): ds/dt = Omega x s, time-centred momentum */
    if (fl & ORC_F_TBMT) {
        double pb[3] = {0.5 * (pold[0] + p[0]), 0.5 * (pold[1] + p[1]), 0.5 * (pold[2] + p[2])};
        double gb = sqrt(1.0 + dot3(pb, pb));
        double bb[3] = {pb[0] / gb, pb[1] / gb, pb[2] / gb};
        double bB = dot3(bb, B);
        double bxE[3];
        cross3(bb, E, bxE);
        double Om[3];
        /* anomalous moment: alpha/(2 pi); g(chi) with chi of the time-centred momentum (Sec. 8.6.2);
         * none (g = 2) for the comparison run, or when the loop's Scorer term carries it */
        double aT = aE;
        if (fl & (ORC_F_G2 | ORC_F_LOOP)) aT = 0.0;
        else if (fl & ORC_F_AMM) aT = orc_amm_lookup(tb, chi_of(fd->eta0, gb, pb, E, B));
        if (fl & ORC_F_TBMT_PAPER) {
            /* as printed: (a + 1/gamma)(B - v x E) - (a gamma/(gamma+1))(v.B) v */
            for (int i = 0; i < 3; ++i)
                Om[i] = -q * ((aT + 1.0 / gb) * (B[i] - bxE[i]) - (aT * gb / (gb + 1.0)) * bB * bb[i]);
        } else {
            /* standard (Jackson 11.170): (a + 1/gamma) B - (a gamma/(gamma+1))(beta.B) beta - (a + 1/(gamma+1)) beta x E */
            for (int i = 0; i < 3; ++i)
                Om[i] = -q * ((aT + 1.0 / gb) * B[i] - (aT * gb / (gb + 1.0)) * bB * bb[i] - (aT + 1.0 / (gb + 1.0)) * bxE[i]);
        }
        double om = sqrt(dot3(Om, Om));
        if (om > 0.0) {
            double n[3] = {Om[0] / om, Om[1] / om, Om[2] / om};
            rotate(s, n, om * dt);
        }
    }

    double gam = sqrt(1.0 + dot3(p, p));
    if (fl & ORC_F_MOVE)
        for (int i = 0; i < 3; ++i) x[i] += p[i] / gam * dt;

    int event = 0;
    double pf[3] = {p[0], p[1], p[2]};
    double sf[3] = {s[0], s[1], s[2]};
    double tauf = tau;
    if (fl & ORC_F_EMIT) {
        double chi = chi_of(fd->eta0, gam, p, E, B);
        double pn = sqrt(dot3(p, p));
        double khat[3], eps[3], beta[3];
        int ok = pn > 0.0 && chi >= st->chi_floor && chi > 0.0;
        if (ok) {
            for (int i = 0; i < 3; ++i) khat[i] = p[i] / pn;
            double v[3] = {p[0] / gam, p[1] / gam, p[2] / gam};
            ok = make_basis(E, B, v, khat, -(double)q, eps, beta);
        }
        if (ok) {
            int cl = 0;
            double pref = ORC_ALPHA / (ORC_SQRT3 * ORC_PI * fd->eta0 * gam);
            double Wu = pref * orc_nlc_rate_lookup(tb, 0, chi, &cl);
            double Wd = pref * orc_nlc_rate_lookup(tb, 1, chi, NULL);
            res->clamped = cl;
            int resolved = (fl & ORC_F_RESOLVED) != 0;
            double sb = resolved ? dot3(s, beta) : 0.0;
            /* Sec. 5.1: W_s = W_up (1 + s.beta)/2 + W_down (1 - s.beta)/2 */
            double Wup_part = Wu * (1.0 + sb) / 2.0, Wdn_part = Wd * (1.0 - sb) / 2.0;
            double Ws = Wup_part + Wdn_part;
            double u0[2];
            int down = 0;
            double rej_up = 0.0;
            if (fl & ORC_F_REJECT) {
                /* table-free (Sec. 4.2): rejection with the proposal f = r^3.  The candidate energy
                 * fraction lambda = r1^3 is accepted if r2 < 3 r1^2 (dW/dlambda)(lambda) dt, with
                 * dW/dlambda = pref w(lambda; s.beta) the spin-resolved density (App. A.1); the
                 * acceptance must stay below 1 (counted when it does not); no optical depth */
                orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_TAU_BRANCH, u0);
                double lc = u0[0] * u0[0] * u0[0], om = 1.0 - lc;
                rej_up = 2.0 * lc / (3.0 * chi * om);
                double b[3];
                orc_bessel(rej_up, b);
                double wl = -b[2] + (1.0 / om + om) * b[1] + lc * sb * b[0];
                double acc = 3.0 * u0[0] * u0[0] * pref * wl * dt;
                res->bound = acc > 1.0;
                event = u0[1] < acc;
            } else if (fl & ORC_F_TAU) {
                /* optical depth (Sec. 4.1): tau_rem decreases by W dt, event when <= 0 */
                tauf = tau - Ws * dt;
                event = tauf <= 0.0;
                if (event) {
                    orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_TAU_BRANCH, u0);
                    /* branch with a fresh r_b: down if r_b W_s < W_down (1 - s.beta)/2 */
                    down = u0[1] * Ws < Wdn_part;
                }
            } else {
                /* per-step probability (Sec. 4.1, 5.1): event if r1 < W_s dt; down if r1 < W_down (1-s.beta) dt/2 */
                orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_TAU_BRANCH, u0);
                event = u0[0] < Ws * dt;
                down = u0[0] < Wdn_part * dt;
            }
            if (event) {
                /* the state the classical part of the step gave the lepton, with its optical depth
                 * spent: what it keeps if its photon finds no room in the photon buffer */
                for (int i = 0; i < 3; ++i) { res->kept_p[i] = p[i]; res->kept_s[i] = s[i]; }
                res->kept_tau = tauf;
                double u1[2], u2[2];
                orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_LAMBDA_SPIN, u1);
                orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_STOKES, u2);
                /* lambda from the ICDF of the chosen branch (Sec. 5.1), or the accepted candidate, or
                 * (the learned sampler's target) the exact quantile of the mixture w(lambda; s.beta) at
                 * the same r2: the branch pair samples that mixture, so both draw one distribution */
                double up;
                if (fl & ORC_F_REJECT) {
                    up = rej_up;
                } else if (fl & ORC_F_MIX_QUANTILE) {
                    double o[4];
                    orc_mlp_target(chi, u1[0], sb, o);
                    up = exp(o[0]);
                } else {
                    up = exp(orc_icdf_lookup(tb, 0, down ? 1 : 0, chi, u1[0]));
                }
                double lam = orc_nlc_lambda(chi, up);
                /* photon and recoil (Sec. 5.1): hbar k = lambda p_i, p_f = (1 - lambda) p_i */
                double k[3] = {lam * p[0], lam * p[1], lam * p[2]};
                if (fl & ORC_F_RECOIL)
                    for (int i = 0; i < 3; ++i) pf[i] = (1.0 - lam) * p[i];
                double bes[3];
                orc_bessel_scaled(up, bes); /* common factor e^{-u'} cancels in g/w and F/F0 */
                double si[3] = {0.0, 0.0, 0.0}, sfu[3] = {0.0, 0.0, 0.0}, xi[3] = {0.0, 0.0, 0.0};
                if (resolved) for (int i = 0; i < 3; ++i) si[i] = s[i];
                if (fl & ORC_F_SPIN_EVENT) {
                    double w, g[3];
                    orc_nlc_wg(lam, bes, si, eps, beta, khat, &w, g);
                    double gn = sqrt(dot3(g, g));
                    if (fl & ORC_F_BETA_BASIS) {
                        /* beta basis (Sec. 8.3): the final spin resolved along +-beta only; the probability
                         * of -beta is (w - g.beta)/(2w), the expectation (g.beta/w) beta */
                        double gb = dot3(g, beta);
                        if (fl & ORC_F_SPIN_COLLAPSE) {
                            double sg = u1[1] < (w - gb) / (2.0 * w) ? -1.0 : 1.0;
                            for (int i = 0; i < 3; ++i) sf[i] = sg * beta[i];
                        } else {
                            for (int i = 0; i < 3; ++i) sf[i] = gb / w * beta[i];
                        }
                    } else if (fl & ORC_F_SPIN_COLLAPSE) {
                        /* SQA collapse (Sec. 5.1): s_f = -S if r3 < (w - |g|)/(2w), else +S */
                        double sg = u1[1] < (w - gn) / (2.0 * w) ? -1.0 : 1.0;
                        for (int i = 0; i < 3; ++i) sf[i] = gn > 0.0 ? sg * g[i] / gn : 0.0;
                    } else {
                        for (int i = 0; i < 3; ++i) sf[i] = g[i] / w;
                    }
                    for (int i = 0; i < 3; ++i) sfu[i] = sf[i];
                }
                if (fl & ORC_F_POL_EVENT) {
                    /* photon Stokes given (s_i, s_f) (Sec. 5.1, App. A.1); s_f = 0 sums over final spins */
                    double F[4];
                    orc_nlc_stokes(lam, bes, si, sfu, eps, beta, khat, F);
                    double Fn = sqrt(F[1] * F[1] + F[2] * F[2] + F[3] * F[3]);
                    if (fl & ORC_F_POL_COLLAPSE) {
                        /* PQA collapse: xi = -Xi if r4 < (F0 - |F|)/(2 F0), else +Xi */
                        double sg = u2[0] < (F[0] - Fn) / (2.0 * F[0]) ? -1.0 : 1.0;
                        for (int i = 0; i < 3; ++i) xi[i] = Fn > 0.0 ? sg * F[i + 1] / Fn : 0.0;
                    } else {
                        for (int i = 0; i < 3; ++i) xi[i] = F[i + 1] / F[0];
                    }
                }
                double P[3];
                orc_stokes_to_P(xi, eps, beta, khat, P);
                /* new optical depth for the emitter */
                if ((fl & ORC_F_TAU) && !(fl & ORC_F_REJECT)) tauf = -log(u0[0]);
                res->event = 1;
                double kn = sqrt(dot3(k, k));
                res->store = kn >= st->photon_store_min;
                uint64_t cid[2];
                orc_child_ids(id, st->seed, st->step, cid);
                res->id0 = cid[0];
                for (int i = 0; i < 3; ++i) { res->d0[i] = x[i]; res->k0[i] = k[i]; res->P0[i] = P[i]; }
                res->tau0 = orc_birth_tau(cid[0], st->seed);
                res->w0 = L->w[j];
            } else if ((fl & ORC_F_NONTRANSITION) && resolved) {
                /* Sec. 6: s <- [s (1 - <P> dt) - P_i dt] / [1 - (<P> + P_i . s) dt],
                 * <P> = (W_up + W_down)/2, P_i = ((W_up - W_down)/2) beta */
                double W0 = 0.5 * (Wu + Wd), Pi = 0.5 * (Wu - Wd);
                double D = 1.0 - (W0 + Pi * dot3(beta, s)) * dt;
                if (D > 0.0) {
                    for (int i = 0; i < 3; ++i) sf[i] = (s[i] * (1.0 - W0 * dt) - Pi * beta[i] * dt) / D;
                    double n2 = dot3(sf, sf);
                    if (n2 > 1.0) {
                        double n = sqrt(n2);
                        for (int i = 0; i < 3; ++i) sf[i] /= n;
                        res->renorm = 1;
                    }
                }
            }
            if (!event && (fl & ORC_F_LOOP)) {
                /* Scorer term of the loop Mueller matrix (App. A.1, R_if): the antisymmetric part in the
                 * (k, eps) plane turns the spin about the rest-frame magnetic field, at a(chi) times the
                 * rest-frame field chi/eta0, in the lepton's proper time (1/gamma per unit lab time), with
                 * the T-BMT sense (-q).  B' = gamma (B - v x E) - gamma^2/(gamma+1) (v.B) v. */
                double v[3] = {p[0] / gam, p[1] / gam, p[2] / gam};
                double vxE[3];
                cross3(v, E, vxE);
                double vB = dot3(v, B), Bp[3];
                for (int i = 0; i < 3; ++i) Bp[i] = gam * (B[i] - vxE[i]) - gam * gam / (gam + 1.0) * vB * v[i];
                double nb = sqrt(dot3(Bp, Bp));
                if (nb > 0.0) {
                    double n[3] = {-q * Bp[0] / nb, -q * Bp[1] / nb, -q * Bp[2] / nb};
                    rotate(sf, n, orc_amm_lookup(tb, chi) * chi / (fd->eta0 * gam) * dt);
                }
            }
        }
    }
    L->x[j] = x[0]; L->y[j] = x[1]; L->z[j] = x[2];
    L->px[j] = pf[0]; L->py[j] = pf[1]; L->pz[j] = pf[2];
    L->sx[j] = sf[0]; L->sy[j] = sf[1]; L->sz[j] = sf[2];
    L->tau[j] = tauf;
}

int orc_lepton_step(const orc_tables *tb, const orc_field *fd, const orc_step *st, int32_t charge,
                    orc_particles *L, orc_particles *ph, orc_counters *ctr)
{
    int64_t n = L->n;
    /* g(chi) and the loop term need the a(chi) table; a(chi) in T-BMT and the loop's Scorer term are the
     * same anomalous moment, and g = 2 excludes both */
    if ((st->flags & (ORC_F_AMM | ORC_F_LOOP)) && !tb->amm) return -2;
    if ((st->flags & ORC_F_AMM) && (st->flags & (ORC_F_LOOP | ORC_F_G2))) return -2;
    orc_result *res = (orc_result *)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_result));
    if (!res) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) lepton_one(tb, fd, st, charge, L, j, &res[j]);
    /* daughters appended in parent order (Sec. 4.3).  An event whose photon does not fit is not applied:
     * the lepton keeps the state the classical part of its step gave it and its spent optical depth, so
     * it emits in a later step (without a photon buffer the photons are discarded and events apply). */
    for (int64_t j = 0; j < n; ++j) {
        if (res[j].clamped) ctr->chi_clamped++;
        if (res[j].renorm) ctr->renormalised++;
        if (res[j].bound) ctr->bound_exceeded++;
        if (!res[j].event) continue;
        if (!res[j].store) { ctr->events++; ctr->below_store++; continue; }
        if (ph == NULL) { ctr->events++; ctr->dropped_capacity++; continue; }
        if (ph->n >= ph->capacity) {
            ctr->dropped_capacity++;
            L->px[j] = res[j].kept_p[0]; L->py[j] = res[j].kept_p[1]; L->pz[j] = res[j].kept_p[2];
            L->sx[j] = res[j].kept_s[0]; L->sy[j] = res[j].kept_s[1]; L->sz[j] = res[j].kept_s[2];
            L->tau[j] = res[j].kept_tau;
            continue;
        }
        ctr->events++;
        push_particle(ph, res[j].d0, res[j].k0, res[j].P0, res[j].tau0, res[j].w0, res[j].id0);
        ctr->stored++;
    }
    free(res);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Photon step: ballistic move and the NBW module (Sec. 5.2 and its flow chart;*/
/* non-pair update Sec. 6).                                                    */
/* ------------------------------------------------------------------------- */
static void photon_one(const orc_tables *tb, const orc_field *fd, const orc_step *st, orc_particles *G, int64_t j,
                       orc_result *res)
{
    const uint32_t fl = st->flags;
    const double dt = st->dt;
    memset(res, 0, sizeof(*res));
    double x[3] = {G->x[j], G->y[j], G->z[j]};
    double k[3] = {G->px[j], G->py[j], G->pz[j]};
    double P[3] = {G->sx[j], G->sy[j], G->sz[j]};
    double tau = G->tau[j];
    uint64_t id = G->id[j];
    double E[3], B[3];
    orc_field_eval(fd, x, st->t, E, B); /* fields at the pre-move position */
    double en = sqrt(dot3(k, k));
    double khat[3] = {0, 0, 0};
    if (en > 0.0)
        for (int i = 0; i < 3; ++i) khat[i] = k[i] / en;
    if (fl & ORC_F_MOVE)
        for (int i = 0; i < 3; ++i) x[i] += khat[i] * dt;
    double Pf[3] = {P[0], P[1], P[2]};
    double tauf = tau;
    if ((fl & ORC_F_EMIT) && en > 0.0) {
        double chi = chi_of(fd->eta0, en, k, E, B);
        double eps[3], beta[3];
        int ok = chi >= st->chi_floor && chi > 0.0 && make_basis(E, B, khat, khat, 1.0, eps, beta);
        if (ok) {
            int resolved = (fl & ORC_F_RESOLVED) != 0;
            double xi[3];
            orc_P_to_stokes(P, eps, beta, khat, xi);
            if (!resolved) xi[0] = xi[1] = xi[2] = 0.0;
            int cl = 0;
            double pref = ORC_ALPHA / (ORC_SQRT3 * ORC_PI * fd->eta0 * en);
            double Wp = pref * orc_nbw_rate_lookup(tb, 0, chi, &cl);
            double Wm = pref * orc_nbw_rate_lookup(tb, 1, chi, NULL);
            res->clamped = cl;
            /* Sec. 5.2: W_xi = W_- (1 - xi3)/2 + W_+ (1 + xi3)/2 */
            double Wm_part = Wm * (1.0 - xi[2]) / 2.0, Wp_part = Wp * (1.0 + xi[2]) / 2.0;
            double Wx = Wm_part + Wp_part;
            int event = 0, minus = 0;
            double u0[2];
            double rej_lam = 0.0, rej_ut = 0.0;
            if (fl & ORC_F_REJECT) {
                /* table-free (Sec. 4.2): the pair spectrum is bounded, so the candidate positron fraction
                 * is lambda = r1 itself, accepted if r2 < (dW/dlambda)(lambda) dt = pref w0(lambda; xi3) dt
                 * (App. A.2); no optical depth */
                orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_TAU_BRANCH, u0);
                double lc = u0[0], om = 1.0 - u0[0];
                rej_lam = lc;
                rej_ut = 2.0 / (3.0 * chi * lc * om);
                double b[3];
                orc_bessel(rej_ut, b);
                double w0 = b[2] + (om / lc + lc / om) * b[1] - xi[2] * b[1];
                double acc = pref * w0 * dt;
                res->bound = acc > 1.0;
                event = u0[1] < acc;
            } else if (fl & ORC_F_TAU) {
                tauf = tau - Wx * dt;
                event = tauf <= 0.0;
                if (event) {
                    orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_TAU_BRANCH, u0);
                    minus = u0[1] * Wx < Wm_part;
                }
            } else {
                orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_TAU_BRANCH, u0);
                event = u0[0] < Wx * dt;
                minus = u0[0] < Wm_part * dt;
            }
            if (event && ((fl & ORC_F_REJECT) || Wx > 0.0)) {
                double u1[2];
                orc_uniform_pair(id, st->seed, st->step, ORC_SLOT_LAMBDA_SPIN, u1);
                double lam, ut;
                if (fl & ORC_F_REJECT) {
                    lam = rej_lam;
                    ut = rej_ut;
                } else {
                    /* lambda from the folded ICDF of the chosen branch (Sec. 5.2) */
                    double r = u1[0];
                    double rf = r < 0.5 ? 1.0 - 2.0 * r : 2.0 * r - 1.0;
                    double xv;
                    if (rf > 0.0) xv = exp(orc_icdf_lookup(tb, 1, minus ? 1 : 0, chi, rf));
                    else xv = 0.0;
                    double mu = orc_nbw_mu(chi, xv);
                    lam = r < 0.5 ? mu : 1.0 - mu;
                    ut = 8.0 / (3.0 * chi) + xv;
                }
                double bes[3];
                orc_bessel_scaled(ut, bes);
                double pe[3], pp[3];
                for (int i = 0; i < 3; ++i) { pp[i] = lam * k[i]; pe[i] = (1.0 - lam) * k[i]; }
                double se[3] = {0, 0, 0}, sp[3] = {0, 0, 0};
                if (fl & ORC_F_SPIN_EVENT) {
                    double w0, je[3], jp[3];
                    orc_nbw_j(lam, bes, xi, eps, beta, khat, &w0, je, jp);
                    if (fl & ORC_F_SPIN_COLLAPSE) {
                        double jen = sqrt(dot3(je, je)), jpn = sqrt(dot3(jp, jp));
                        double Se[3], Sp[3];
                        for (int i = 0; i < 3; ++i) {
                            Se[i] = jen > 0.0 ? je[i] / jen : 0.0;
                            Sp[i] = jpn > 0.0 ? jp[i] / jpn : 0.0;
                        }
                        /* beta basis: both axes beta (the four G_ab still sum to 4 w0 for any axes) */
                        if (fl & ORC_F_BETA_BASIS)
                            for (int i = 0; i < 3; ++i) { Se[i] = beta[i]; Sp[i] = beta[i]; }
                        /* four correlated states (Sec. 5.2), order (--, -+, +-, ++), first sign = positron,
                         * probabilities G_ab / (4 w0) */
                        double cum = 0.0;
                        int chosen = 3;
                        for (int a = 0; a < 4; ++a) {
                            double sa = (a & 2) ? 1.0 : -1.0, sbb = (a & 1) ? 1.0 : -1.0;
                            double spv[3] = {sa * Sp[0], sa * Sp[1], sa * Sp[2]};
                            double sev[3] = {sbb * Se[0], sbb * Se[1], sbb * Se[2]};
                            double Gv[4];
                            orc_nbw_G(lam, bes, spv, sev, eps, beta, khat, Gv);
                            double Gab = Gv[0] + xi[0] * Gv[1] + xi[1] * Gv[2] + xi[2] * Gv[3];
                            cum += Gab / (4.0 * w0);
                            if (u1[1] < cum) { chosen = a; break; }
                        }
                        double sa = (chosen & 2) ? 1.0 : -1.0, sbb = (chosen & 1) ? 1.0 : -1.0;
                        for (int i = 0; i < 3; ++i) { sp[i] = sa * Sp[i]; se[i] = sbb * Se[i]; }
                    } else if (fl & ORC_F_BETA_BASIS) {
                        double eb = dot3(je, beta) / w0, pb = dot3(jp, beta) / w0;
                        for (int i = 0; i < 3; ++i) { se[i] = eb * beta[i]; sp[i] = pb * beta[i]; }
                    } else {
                        for (int i = 0; i < 3; ++i) { se[i] = je[i] / w0; sp[i] = jp[i] / w0; }
                    }
                }
                uint64_t cid[2];
                orc_child_ids(id, st->seed, st->step, cid);
                res->event = 1;
                res->store = 1;
                res->id0 = cid[0];
                res->id1 = cid[1];
                for (int i = 0; i < 3; ++i) {
                    res->d0[i] = x[i];
                    res->k0[i] = pe[i];
                    res->P0[i] = se[i];
                    res->d1k[i] = pp[i];
                    res->s1[i] = sp[i];
                }
                res->tau0 = orc_birth_tau(cid[0], st->seed);
                res->tau1 = orc_birth_tau(cid[1], st->seed);
                res->w0 = G->w[j];
            } else if (!event && (fl & ORC_F_NONTRANSITION) && resolved) {
                /* Sec. 6 with Q = e3 in Stokes space: xi <- [xi (1 - <P> dt) - P_i dt] / [1 - (<P> + P_i . xi) dt],
                 * <P> = (W_+ + W_-)/2, P_i = ((W_+ - W_-)/2) e3 */
                double W0 = 0.5 * (Wp + Wm), Pi = 0.5 * (Wp - Wm);
                double D = 1.0 - (W0 + Pi * xi[2]) * dt;
                if (D > 0.0) {
                    double xn[3] = {xi[0] * (1.0 - W0 * dt) / D, xi[1] * (1.0 - W0 * dt) / D,
                                    (xi[2] * (1.0 - W0 * dt) - Pi * dt) / D};
                    double n2 = xn[0] * xn[0] + xn[1] * xn[1] + xn[2] * xn[2];
                    if (n2 > 1.0) {
                        double nn = sqrt(n2);
                        for (int i = 0; i < 3; ++i) xn[i] /= nn;
                        res->renorm = 1;
                    }
                    orc_stokes_to_P(xn, eps, beta, khat, Pf);
                }
            }
        }
    }
    G->x[j] = x[0]; G->y[j] = x[1]; G->z[j] = x[2];
    G->sx[j] = Pf[0]; G->sy[j] = Pf[1]; G->sz[j] = Pf[2];
    G->tau[j] = tauf;
}

/* Photons that convert are removed (Sec. 4.3, 5.2); the surviving photons keep
 * their order, daughters are appended in parent order, electron then positron. */
int orc_photon_step(const orc_tables *tb, const orc_field *fd, const orc_step *st, orc_particles *G,
                    orc_particles *el, orc_particles *po, orc_counters *ctr)
{
    int64_t n = G->n;
    orc_result *res = (orc_result *)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_result));
    if (!res) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) photon_one(tb, fd, st, G, j, &res[j]);
    int64_t keep = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (res[j].clamped) ctr->chi_clamped++;
        if (res[j].renorm) ctr->renormalised++;
        if (res[j].bound) ctr->bound_exceeded++;
        int dead = 0;
        if (res[j].event) {
            if (el == NULL || po == NULL || el->n >= el->capacity || po->n >= po->capacity) {
                ctr->dropped_capacity++; /* the photon survives and retries next step */
            } else {
                ctr->events++;
                push_particle(el, res[j].d0, res[j].k0, res[j].P0, res[j].tau0, res[j].w0, res[j].id0);
                push_particle(po, res[j].d0, res[j].d1k, res[j].s1, res[j].tau1, res[j].w0, res[j].id1);
                ctr->stored += 2;
                dead = 1;
            }
        }
        if (!dead) {
            if (keep != j) {
                G->x[keep] = G->x[j]; G->y[keep] = G->y[j]; G->z[keep] = G->z[j];
                G->px[keep] = G->px[j]; G->py[keep] = G->py[j]; G->pz[keep] = G->pz[j];
                G->sx[keep] = G->sx[j]; G->sy[keep] = G->sy[j]; G->sz[keep] = G->sz[j];
                G->tau[keep] = G->tau[j]; G->w[keep] = G->w[j]; G->id[keep] = G->id[j];
            }
            ++keep;
        }
    }
    G->n = keep;
    free(res);
    return 0;
}

/* Optical depth at birth for particles [0, n): tau = -ln u(id, reserved step, slot 0). */
void orc_init_tau(orc_particles *b, uint64_t seed)
{
    for (int64_t j = 0; j < b->n; ++j) b->tau[j] = orc_birth_tau(b->id[j], seed);
}

/* Sokolov-Ternov / BKS functions (Sec. 8.1, 8.3), u'' = u^2/(1+u)^3, argument 2u/(3 chi):
 *   psi1 = int u'' K23,  psi3 = int u'' K13,  psi2 = int u'' IntK13 - psi1.
 * which = 1, 2, 3.  Variable u = v^3 / (1 - v) style map not needed: substitute u = t^3
 * and integrate in t over panels until the integrand is negligible. */
double orc_psi(double chi, int which)
{
    gl_init();
    double s = 0.0;
    double tmax = cbrt(60.0 * 1.5 * chi) + 6.0;
    int np = (int)ceil(tmax / ORC_PANEL_W);
    for (int p = 0; p < np; ++p) {
        double a = p * ORC_PANEL_W, b = (p + 1) * ORC_PANEL_W;
        double m = 0.5 * (a + b), r = 0.5 * (b - a), seg = 0.0;
        for (int i = 0; i < gl_n; ++i) {
            double t = m + r * gl_x[i];
            double u = t * t * t;
            double upp = u * u / ((1.0 + u) * (1.0 + u) * (1.0 + u));
            double bes[3];
            orc_bessel(2.0 * u / (3.0 * chi), bes);
            double f = which == 1 ? bes[1] : which == 3 ? bes[0] : bes[2] - bes[1];
            seg += gl_w[i] * upp * f * 3.0 * t * t;
        }
        s += seg * r;
    }
    return s;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Target of the learned sampler.  Sec. 5.1 samples the photon energy from    */
/* the spin-resolved spectrum w(lambda; s_beta) and notes that a direct table */
/* in (chi, r, s_beta) costs memory; a small network stands in for that 3-D   */
/* inverse CDF.  Its target, written out from the definition:                 */
/*   the r-quantile of w(lambda; s) in u' (t = u'^{1/3}):                      */
/*     C_s(t) = int_0^t [w(s) d lambda/dt'] dt' / int_0^T [...] dt',           */
/*     w(s) = -IntK13 + kappa K23 + lambda s K13  (linear in s, so the blend   */
/*     of the two branch integrands with weights (1 +- s)/2);                  */
/*   the photon Stokes vector at that lambda, final lepton spin summed         */
/*   (s_f = 0), initial spin s_i = s beta_hat, basis eps = x, beta = y, k = z: */
/*     xi_i = F_i / F_0 (App. A.1).                                            */
/* out = {ln u', xi1, xi2, xi3}.  The exact mixture CDF at u' is              */
/* orc_mlp_cdf.                                                                */
/* ------------------------------------------------------------------------- */
static double mix_integrand_t(double chi, double s, double t)
{
    return 0.5 * (1.0 + s) * nlc_integrand_t(chi, 1, t) + 0.5 * (1.0 - s) * nlc_integrand_t(chi, -1, t);
}

static double mix_segment(double chi, double s, double a, double b)
{
    gl_init();
    double m = 0.5 * (a + b), r = 0.5 * (b - a), acc = 0.0;
    for (int i = 0; i < gl_n; ++i) acc += gl_w[i] * mix_integrand_t(chi, s, m + r * gl_x[i]);
    return acc * r;
}

/* exact C_s at u' (the quantity the learned sampler's check compares with r) */
double orc_mlp_cdf(double chi, double s, double ln_up)
{
    double T = t_end(0), t = exp(ln_up / 3.0), total = 0.0, part = 0.0;
    int np = (int)ceil(T / ORC_PANEL_W);
    for (int p = 0; p < np; ++p) {
        double a = p * ORC_PANEL_W, b = fmin(T, (p + 1) * ORC_PANEL_W);
        double seg = mix_segment(chi, s, a, b);
        total += seg;
        if (b <= t) part += seg;
        else if (a < t) part += mix_segment(chi, s, a, t);
    }
    return part / total;
}

void orc_mlp_target(double chi, double r, double s, double out[4])
{
    double T = t_end(0);
    int np = (int)ceil(T / ORC_PANEL_W);
    double *cum = (double *)malloc(sizeof(double) * (np + 1));
    cum[0] = 0.0;
    for (int p = 0; p < np; ++p) {
        double a = p * ORC_PANEL_W, b = fmin(T, (p + 1) * ORC_PANEL_W);
        cum[p + 1] = cum[p] + mix_segment(chi, s, a, b);
    }
    /* solve C_s(t) = r: the panel that brackets r, then Newton (derivative = integrand) kept in the bracket */
    double target = r * cum[np];
    int p = 0;
    while (p < np - 1 && cum[p + 1] < target) ++p;
    double a = p * ORC_PANEL_W, b = fmin(T, (p + 1) * ORC_PANEL_W), base = cum[p];
    double lo = a, hi = b, t = a + (b - a) * (target - base) / (cum[p + 1] - base);
    for (int it = 0; it < 200; ++it) {
        double f = base + mix_segment(chi, s, a, t) - target;
        if (f > 0) hi = t; else lo = t;
        double tn = t - f / mix_integrand_t(chi, s, t);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (fabs(tn - t) <= 1e-15 * fmax(t, 1e-300) || hi - lo <= 1e-15 * hi) { t = tn; break; }
        t = tn;
    }
    free(cum);
    double up = t * t * t, bes[3], F[4];
    double lam = orc_nlc_lambda(chi, up);
    orc_bessel(up, bes);
    const double si[3] = {0.0, s, 0.0}, sf[3] = {0.0, 0.0, 0.0};
    const double eps[3] = {1.0, 0.0, 0.0}, beta[3] = {0.0, 1.0, 0.0}, k[3] = {0.0, 0.0, 1.0};
    orc_nlc_stokes(lam, bes, si, sf, eps, beta, k, F);
    out[0] = 3.0 * log(t);
    out[1] = F[1] / F[0];
    out[2] = F[2] / F[0];
    out[3] = F[3] / F[0];
}
