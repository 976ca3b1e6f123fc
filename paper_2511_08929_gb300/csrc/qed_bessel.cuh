// qed_bessel.cuh -- modified Bessel functions of the App. A spectra and the table lookups
// (Sec. 5.1, 5.2).  All Bessel values are scaled: e^x K_{1/3}(x), e^x K_{2/3}(x),
// e^x int_x^inf K_{1/3} -- the factor cancels in every ratio the event sampling takes, and the
// rate/CDF integrands put it back explicitly.
//
//  * direct evaluation (table build, and x beyond the table): trapezoid rule on
//    e^x K_nu(x) = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt  (DLMF 10.32.9), and
//    e^x IntK13(x) = int_0^inf exp(-x (cosh t - 1)) cosh(t/3)/cosh t dt, with step
//    h = min(0.2, 0.6/sqrt x) (error ~ exp(-pi^2/h) for small x, exp(-2 pi^2/(h^2 x)) for large x);
//  * x < kBesLo: two terms of each ascending series of I_{+-nu} (K_nu = pi (I_-nu - I_nu)/(2 sin nu pi));
//  * otherwise a table on a uniform grid in ln x (spacing 0.02), interpolated by 8-point Lagrange
//    (FP64 path, ~2e-15) or 4-point Lagrange (FP32 path, ~1e-9).
#pragma once
#include "qed_device.cuh"

namespace qed {

constexpr double kBesLo = 1e-4;   // table start
constexpr double kBesH = 0.02;    // spacing in ln x
constexpr int kBesN = 977;        // nodes: ln x in [ln 1e-4, ln 1e-4 + 976 * 0.02] (x up to 2.97e4)
constexpr double kGamma13 = 2.6789385347077476337;  // Gamma(1/3)
constexpr double kGamma23 = 1.3541179394264004169;  // Gamma(2/3)

// --------------------------------------------------------------------------------------------
// direct trapezoid (FP64)
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void bessel_trapezoid(double x, double out[3]) {
    double T = acosh(1.0 + 46.0 / x);
    T = acosh(1.0 + (46.0 + (2.0 / 3.0) * T) / x);
    const double h = fmin(0.2, 0.6 * rsqrt(x));
    const int n = (int)ceil(T / h);
    double s0 = 0.5, s1 = 0.5, s2 = 0.5;  // t = 0: exp(0) * cosh(0) terms, weight 1/2
    for (int m = 1; m <= n; ++m) {
        const double t = m * h;
        const double sh = sinh(0.5 * t);
        const double e = exp(-x * (2.0 * sh * sh));  // cosh t - 1 = 2 sinh^2(t/2)
        const double c3 = cosh(t / 3.0);
        s0 += e * c3;
        s1 += e * (2.0 * c3 * c3 - 1.0);
        s2 += e * c3 / cosh(t);
    }
    out[0] = s0 * h;
    out[1] = s1 * h;
    out[2] = s2 * h;
}

// --------------------------------------------------------------------------------------------
// small-argument series (any precision)
// --------------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void bessel_series(R x, R out[3]) {
    const R a = R(0.5) * x, a2 = a * a;
    const R pi3 = R(kPi / kSqrt3);
    const R g13 = R(kGamma13), g23 = R(kGamma23);
    const R c1 = cbrt(a);   // a^{1/3}
    const R c2 = c1 * c1;   // a^{2/3}
    const R ex = exp_(x);
    // K13 = pi/sqrt3 [a^-1/3/Gamma(2/3) (1 + a^2/(2/3)) - a^1/3/Gamma(4/3) (1 + a^2/(4/3))]
    out[0] = pi3 * (rcp_(c1 * g23) * (R(1) + R(1.5) * a2) - div_(R(3) * c1, g13) * (R(1) + R(0.75) * a2)) * ex;
    // K23 = pi/sqrt3 [a^-2/3/Gamma(1/3) (1 + a^2/(1/3)) - a^2/3/Gamma(5/3) (1 + a^2/(5/3))]
    out[1] = pi3 * (rcp_(c2 * g13) * (R(1) + R(3) * a2) - div_(R(1.5) * c2, g23) * (R(1) + R(0.6) * a2)) * ex;
    // IntK13 = pi/sqrt3 - int_0^x K13 = pi/sqrt3 [1 - 3 a^2/3/Gamma(2/3) (1 + 3 a^2/8) + 1.5 a^4/3/Gamma(4/3) (1 + 3 a^2/10)]
    out[2] = pi3 * (R(1) - div_(R(3) * c2, g23) * (R(1) + R(0.375) * a2) + div_(R(4.5) * c2 * c2, g13) * (R(1) + R(0.3) * a2)) * ex;
}

// --------------------------------------------------------------------------------------------
// table interpolation
// --------------------------------------------------------------------------------------------
// FP64: tab[3][kBesN] of scaled values.
__device__ __forceinline__ void bessel64(const double* __restrict__ tab, double x, double out[3]) {
    if (x < kBesLo) {
        bessel_series<double>(x, out);
        return;
    }
    const double t = (log(x) - log(kBesLo)) / kBesH;
    if (t > kBesN - 1) {
        bessel_trapezoid(x, out);
        return;
    }
    int j0 = (int)floor(t);
    if (j0 < 3) j0 = 3;
    if (j0 > kBesN - 5) j0 = kBesN - 5;
    const double tau = t - j0;
    // Lagrange weights on nodes m = -3..4: L_k = prod_{m != k} (tau - m)/(k - m)
    double d[8], pre[8], suf[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = tau - (i - 3);
    pre[0] = 1.0;
#pragma unroll
    for (int i = 1; i < 8; ++i) pre[i] = pre[i - 1] * d[i - 1];
    suf[7] = 1.0;
#pragma unroll
    for (int i = 6; i >= 0; --i) suf[i] = suf[i + 1] * d[i + 1];
    // 1 / prod_{m != k}(k - m) for k = -3..4
    const double c[8] = {-1.0 / 5040.0, 1.0 / 720.0, -1.0 / 240.0, 1.0 / 144.0, -1.0 / 144.0, 1.0 / 240.0, -1.0 / 720.0,
                         1.0 / 5040.0};
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const double L = pre[i] * suf[i] * c[i];
        const int j = j0 - 3 + i;
        v0 += L * tab[j];
        v1 += L * tab[kBesN + j];
        v2 += L * tab[2 * kBesN + j];
    }
    out[0] = v0;
    out[1] = v1;
    out[2] = v2;
}

// FP32: tab[3][kBesN] floats (shared memory in the step kernels); beyond the table the leading
// large-x asymptotics sqrt(pi/(2x)) (1 + c/x).
__device__ __forceinline__ void bessel32(const float* tab, float x, float out[3]) {
    if (x < float(kBesLo)) {
        bessel_series<float>(x, out);
        return;
    }
    const float t = (__logf(x) - float(-9.210340371976182)) * float(1.0 / kBesH);  // ln(1e-4)
    if (t > float(kBesN - 1)) {
        const float ix = rcp_(x), a = sqrt_(float(kPi / 2.0) * ix);
        out[0] = a * (1.0f - (5.0f / 72.0f) * ix);   // (4 nu^2 - 1)/8 with nu = 1/3
        out[1] = a * (1.0f + (7.0f / 72.0f) * ix);   // nu = 2/3
        out[2] = a * (1.0f - (41.0f / 72.0f) * ix);  // int_x^inf: (4 nu^2 - 5)/8
        return;
    }
    int j0 = (int)t;
    if (j0 < 1) j0 = 1;
    if (j0 > kBesN - 3) j0 = kBesN - 3;
    const float tau = t - (float)j0;
    const float wm1 = -tau * (tau - 1.0f) * (tau - 2.0f) * (1.0f / 6.0f);
    const float w0 = (tau + 1.0f) * (tau - 1.0f) * (tau - 2.0f) * 0.5f;
    const float w1 = -(tau + 1.0f) * tau * (tau - 2.0f) * 0.5f;
    const float w2 = (tau + 1.0f) * tau * (tau - 1.0f) * (1.0f / 6.0f);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const float* r = tab + f * kBesN + j0;
        out[f] = wm1 * r[-1] + w0 * r[0] + w1 * r[1] + w2 * r[2];
    }
}

// --------------------------------------------------------------------------------------------
// rate / ICDF lookups (the interpolation rules are part of the tables' definition, see qed.h)
// --------------------------------------------------------------------------------------------
template <class R>
struct TabP {
    const R* nlc_rate;  // [2][n_chi]
    const R* nbw_rate;  // [2][n_chi]
    const R* nlc_icdf;  // [2][n_chi][n_r]
    const R* nbw_icdf;  // [2][n_chi][n_r]
    const R* nlc_icdf_lo;  // FP32 only: nlc_icdf's rounding remainders (entry = nlc_icdf + nlc_icdf_lo)
    const R* amm;       // [n_chi] ln a(chi), the field-dependent anomalous moment
    R lnchi_min, inv_dlnchi, chi_min, chi_max;
    R y_lo, inv_dy, inv_dy_lo;  // inv_dy + inv_dy_lo: (n_r - 1)/(y_hi - y_lo) to twice the precision of R
    int n_chi, n_r;
};

// chi row coordinate (i, f): linear in ln chi, clamped to the grid
template <class R>
__device__ __forceinline__ void chi_coord(const TabP<R>& T, R lnchi, int& i, R& f) {
    const R s = (lnchi - T.lnchi_min) * T.inv_dlnchi;
    const bool below = !(s > R(0)), above = s >= R(T.n_chi - 1);
    int k = (int)(below || above ? R(0) : s);  // selects, not branches: lanes differ in chi
    if (k > T.n_chi - 2) k = T.n_chi - 2;
    const R fk = s - R(k);
    i = below ? 0 : (above ? T.n_chi - 2 : k);
    f = below ? R(0) : (above ? R(1) : fk);
}

// NLC rate integrals I_up, I_down at chi (classical chi-proportional below chi_min, clamped above chi_max)
template <class R>
__device__ __forceinline__ void nlc_rates(const TabP<R>& T, R chi, R lnchi, R& Iu, R& Id) {
    if (chi < T.chi_min) {
        const R sc = div_(chi, T.chi_min);
        Iu = exp_(T.nlc_rate[0]) * sc;
        Id = exp_(T.nlc_rate[T.n_chi]) * sc;
        return;
    }
    int i; R f;
    chi_coord(T, lnchi, i, f);
    Iu = exp_(fma_(f, T.nlc_rate[i + 1] - T.nlc_rate[i], T.nlc_rate[i]));
    Id = exp_(fma_(f, T.nlc_rate[T.n_chi + i + 1] - T.nlc_rate[T.n_chi + i], T.nlc_rate[T.n_chi + i]));
}

// field-dependent anomalous moment a(chi) (one-loop Scorer term, App. A.1; Sec. 8.6.2): linear in
// (ln chi, ln a) between nodes, the end values outside the grid (chi <= 0 reads the first node)
template <class R>
__device__ __forceinline__ R amm_lookup(const TabP<R>& T, R chi) {
    int i; R f;
    chi_coord(T, chi > R(0) ? log_(chi) : T.lnchi_min, i, f);
    return exp_(fma_(f, T.amm[i + 1] - T.amm[i], T.amm[i]));
}

// the anomalous moment T-BMT precesses with: alpha/(2 pi); a(chi) at the time-centred momentum pb
// (QED_F_AMM); zero for g = 2 (QED_F_G2) and when the loop's Scorer term carries it (QED_F_LOOP)
template <class R>
__device__ __forceinline__ R tbmt_a(uint32_t fl, const TabP<R>& T, R eta0, const V3<R>& pb, const V3<R>& E,
                                    const V3<R>& B) {
    if (fl & (QED_F_G2 | QED_F_LOOP)) return R(0);
    if (fl & QED_F_AMM) return amm_lookup(T, chi_of(eta0, sqrt_(R(1) + dot(pb, pb)), pb, E, B));
    return R(kAlpha / (2.0 * kPi));
}

// the loop's Scorer term in the no-emission update (QED_F_LOOP; App. A.1 R_if): a turn about the
// rest-frame magnetic field B' = gamma (B - v x E) - gamma^2/(gamma+1) (v.B) v by a(chi) chi dt/(eta0 gamma),
// in the T-BMT sense (-q).  Returned as the vector Omega with s <- rotate(s, Omega, dt).
template <class R>
__device__ __forceinline__ V3<R> loop_omega(const TabP<R>& T, R eta0, R chi, R gam, const V3<R>& p, const V3<R>& E,
                                            const V3<R>& B, R q) {
    const R ig = rcp_(gam);
    const V3<R> v = ig * p;
    const V3<R> Bp = axpy(-(div_(gam * gam, gam + R(1)) * dot(v, B)), v, gam * (B - cross(v, E)));
    const R nb2 = dot(Bp, Bp);
    if (!(nb2 > R(0))) return V3<R>{R(0), R(0), R(0)};
    const R rate = amm_lookup(T, chi) * div_(chi, eta0) * ig;
    return ((-q) * rate * rsqrt_(nb2)) * Bp;
}

// NBW rate integrals J_+, J_- at chi (zero below chi_min)
template <class R>
__device__ __forceinline__ void nbw_rates(const TabP<R>& T, R chi, R lnchi, R& Jp, R& Jm) {
    if (chi < T.chi_min) { Jp = R(0); Jm = R(0); return; }
    int i; R f;
    chi_coord(T, lnchi, i, f);
    const R chic = chi > T.chi_max ? T.chi_max : chi;
    const R sub = div_(R(8.0 / 3.0), chic);
    Jp = exp_(fma_(f, T.nbw_rate[i + 1] - T.nbw_rate[i], T.nbw_rate[i]) - sub);
    Jm = exp_(fma_(f, T.nbw_rate[T.n_chi + i + 1] - T.nbw_rate[T.n_chi + i], T.nbw_rate[T.n_chi + i]) - sub);
}

// one ICDF row at logit y: the cubic through the 4 nearest nodes inside the grid (written in Newton form
// about node m: b + x ((c - b) + (x - 1) (D2 + (x + 1) D3)), the same polynomial as the Lagrange form,
// rounding on the small differences), the asymptote below, the last entry above.  The position inside
// the cell is one FMA relative to node m, so it keeps the precision of y.
template <class R>
__device__ __forceinline__ R icdf_row(const R* __restrict__ row, const TabP<R>& T, R slope, R y) {
    const R tt = y * T.inv_dy - T.y_lo * T.inv_dy;
    if (!(tt > R(0))) return row[0] + slope * (y - T.y_lo);
    if (tt >= R(T.n_r - 1)) return row[T.n_r - 1];
    int m = (int)tt;
    if (m < 1) m = 1;
    if (m > T.n_r - 3) m = T.n_r - 3;
    const R x = fma(y, T.inv_dy, -T.y_lo * T.inv_dy - R(m));
    const R a = row[m - 1], b = row[m], c = row[m + 1], d = row[m + 2];
    const R d1 = c - b;
    const R d2 = R(0.5) * ((a - b) + (c - b));
    R d3 = (d - a) + R(3) * (b - c);
    if constexpr (sizeof(R) == 8) d3 = d3 / R(6);
    else d3 = d3 * R(1.0 / 6.0);
    return b + x * (d1 + (x - R(1)) * (d2 + (x + R(1)) * d3));
}

// ln of the sampled variable (NLC: u'; NBW: x) for chi and the uniform r; rows blended in ln chi
template <class R>
__device__ __forceinline__ R icdf_lookup(const TabP<R>& T, bool nbw, int s, R lnchi, R y) {
    const R* base = (nbw ? T.nbw_icdf : T.nlc_icdf) + (size_t)s * T.n_chi * T.n_r;
    int i; R f;
    chi_coord(T, lnchi, i, f);
    const R slope = nbw ? R(2) : R(3);
    const R v0 = icdf_row(base + (size_t)i * T.n_r, T, slope, y);
    const R v1 = icdf_row(base + (size_t)(i + 1) * T.n_r, T, slope, y);
    return v0 + f * (v1 - v0);
}

// --------------------------------------------------------------------------------------------
// the NLC energy fraction of an event to FP32 relative precision (the FP32 path's event pass)
// --------------------------------------------------------------------------------------------
// ln u' of a soft photon is ~ -40; in plain FP32 its rounding (4e-6) would be the relative error of
// the photon's energy.  Here every large quantity is carried as an unevaluated sum of two floats
// (hi exact or exactly rounded, lo the small rest) and only small corrections are rounded: the logit
// y of the uniform from its 52 integer bits, the cell coordinate, the ICDF entries (hi + lo tables),
// and u' = exp(hi) exp(correction).  Relative error of u' ~3e-7.

// a + b = s + e exactly (TwoSum)
__device__ __forceinline__ float two_sum_f(float a, float b, float& e) {
    const float s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
    return s;
}

// ln of u = (m + 1/2) 2^-52 (m = (h20 << 32) | lo, 52 bits) as hi + lo: u = A + B + C exactly with
// A = h20 2^-20, B = (lo & ~0xFF) 2^-52, C = ((lo & 0xFF) + 1/2) 2^-52; s + e = u (TwoSum), s = 2^E M
// with M in [1, 2); ln u = E ln2_hi (exact: ln2_hi has 17 significant bits) + (E ln2_lo + ln M + e/s).
// Also returns u rounded to float.
__device__ __forceinline__ float ln_u52(uint32_t h20, uint32_t lo, float& ln_lo, float& u_f) {
    const float A = (float)h20 * 0x1.0p-20f;
    const float Bv = (float)(lo & 0xFFFFFF00u) * 0x1.0p-52f;
    const float Cv = ((float)(lo & 0xFFu) + 0.5f) * 0x1.0p-52f;
    float e1, e2;
    float s = two_sum_f(A, Bv, e1);
    s = two_sum_f(s, Cv, e2);
    const float e = e1 + e2;
    u_f = s;
    const uint32_t bits = __float_as_uint(s);
    const int E = (int)((bits >> 23) & 0xFFu) - 127;
    const float M = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    const float fE = (float)E;
    ln_lo = fmaf(fE, 1.42860677e-6f, logf(M) + e / s);  // ln 2 = 0.693145752 + 1.42860677e-6
    return fE * 0.693145752f;
}

// y = ln u - ln(1 - u) of the uniform as hi + lo, normalised (|lo| <= ulp(hi)/2); the complementary
// integer for u >= 1/2
__device__ __forceinline__ float logit_u52(uint32_t hi, uint32_t lo, float& y_lo) {
    const uint32_t h20 = hi >> 12;
    const bool upper = h20 >= 0x80000u;  // u >= 1/2: y = -(ln v - ln(1 - v)), v = 1 - u
    float l_lo, uf;
    const float l_hi = upper ? ln_u52(0xFFFFFu - h20, ~lo, l_lo, uf) : ln_u52(h20, lo, l_lo, uf);
    float e;
    const float y = two_sum_f(l_hi, l_lo - log1pf(-uf), e);
    y_lo = upper ? -e : e;
    return upper ? -y : y;
}

// one ICDF row at the cell (m, x) as hi + correction: the cubic through nodes m-1..m+2 (Newton form
// about node m) on hi + lo entries; hi is row[m]'s hi part, the correction carries the rest
__device__ __forceinline__ float icdf_row_ff(const float* __restrict__ rh, const float* __restrict__ rl, int m, float x,
                                             float& corr) {
    const float ah = rh[m - 1], bh = rh[m], ch = rh[m + 1], dh = rh[m + 2];
    const float al = rl[m - 1], bl = rl[m], cl = rl[m + 1], dl = rl[m + 2];
    const float d1 = (ch - bh) + (cl - bl);
    const float d2 = 0.5f * (((ah - bh) + (ch - bh)) + ((al - bl) + (cl - bl)));
    const float d3 = (((dh - ah) + 3.0f * (bh - ch)) + ((dl - al) + 3.0f * (bl - cl))) * (1.0f / 6.0f);
    corr = bl + x * (d1 + (x - 1.0f) * (d2 + (x + 1.0f) * d3));
    return bh;
}

// u' of the NLC ICDF of branch s at lnchi for the uniform of the 52 bits (hi, lo): returns false (and
// nothing) when u' leaves the normal float range, where the caller takes the FP64 lookup
__device__ __forceinline__ bool nlc_up_ff(const TabP<float>& T, int s, float lnchi, uint32_t whi, uint32_t wlo, float& up) {
    float ylo;
    const float yhi = logit_u52(whi, wlo, ylo);
    // cell coordinate tt = (y - y_lo) inv_dy as hi + lo
    float de;
    const float dh = two_sum_f(yhi, -T.y_lo, de);
    const float dl = de + ylo;
    const float tp = dh * T.inv_dy;
    float te;
    const float th = two_sum_f(tp, fmaf(dh, T.inv_dy, -tp) + fmaf(dl, T.inv_dy, dh * T.inv_dy_lo), te);
    const float tl = te;  // th + tl, normalised: the cell index comes from th
    int i;
    float f;
    chi_coord(T, lnchi, i, f);
    const size_t off = (size_t)s * T.n_chi * T.n_r;
    const float* h0 = T.nlc_icdf + off + (size_t)i * T.n_r;
    const float* l0 = T.nlc_icdf_lo + off + (size_t)i * T.n_r;
    const float* h1 = h0 + T.n_r;
    const float* l1 = l0 + T.n_r;
    float base, c0, c1;
    if (!(th + tl > 0.0f)) {  // below the grid: u' ~ r^3, ln u' = row[0] + 3 (y - y_lo)
        const float s3 = 3.0f * dh;
        const float s3e = fmaf(3.0f, dh, -s3);
        float be;
        base = two_sum_f(h0[0], s3, be);
        c0 = be + l0[0] + s3e + 3.0f * dl;
        c1 = (h1[0] - h0[0]) + (l1[0] - l0[0]);
    } else if (th + tl >= (float)(T.n_r - 1)) {  // above the grid: the last entry
        base = h0[T.n_r - 1];
        c0 = l0[T.n_r - 1];
        c1 = (h1[T.n_r - 1] - h0[T.n_r - 1]) + (l1[T.n_r - 1] - l0[T.n_r - 1]);
    } else {
        int m = (int)th;
        if (m < 1) m = 1;
        if (m > T.n_r - 3) m = T.n_r - 3;
        const float x = (th - (float)m) + tl;
        float k0, k1;
        base = icdf_row_ff(h0, l0, m, x, k0);
        const float b1 = icdf_row_ff(h1, l1, m, x, k1);
        c0 = k0;
        c1 = (b1 - base) + (k1 - k0);
    }
    const float corr = fmaf(f, c1, c0);
    if (!(base + corr > -80.0f && base + corr < 80.0f)) return false;
    up = expf(base) * expf(corr);
    return true;
}

}  // namespace qed
