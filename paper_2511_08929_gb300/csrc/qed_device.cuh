// qed_device.cuh -- device building blocks of the spin/polarization-resolved QED step
// (Qian et al., arXiv:2511.08929): counter-based random numbers, analytic fields, the Boris and
// T-BMT pushers, chi and the (eps, beta, k) basis, and the App. A spectra.  Templated on the
// arithmetic type R (double for the plain path, float for the fast path).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qed.h"

namespace qed {

constexpr double kPi = 3.14159265358979323846;
constexpr double kAlpha = 7.2973525693e-3;  // fine-structure constant (CODATA 2018)
constexpr double kSqrt3 = 1.73205080756887729353;
constexpr uint64_t kStepBirth = 0xFFFFFFFFFFFFFFFFull;  // reserved Philox step of a particle's first draw
// Philox counter slot of each draw (counter = (step_lo, step_hi, slot, 0)).
constexpr uint32_t kSlotTauBranch = 0;  // u0: optical depth (or r1 in probability mode), u1: branch r_b
constexpr uint32_t kSlotLambdaSpin = 1; // u0: r2 (energy fraction), u1: r3 (spin collapse)
constexpr uint32_t kSlotStokes = 2;     // u0: r4 (Stokes collapse)
constexpr uint32_t kSlotChild = 3;      // words 0,1 / 2,3: daughter ids

// ---------------------------------------------------------------------------------------------
// small vectors
// ---------------------------------------------------------------------------------------------
template <class R>
struct V3 {
    R x, y, z;
};
template <class R>
__device__ __forceinline__ V3<R> v3(R a, R b, R c) { return V3<R>{a, b, c}; }
// Products and sums are written with explicit fused multiply-adds: one rounding fewer, and the same
// rounding wherever the code is inlined (the FP32 units are built without implicit contraction).
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
template <class R>
__device__ __forceinline__ R dot(const V3<R>& a, const V3<R>& b) { return fma_(a.x, b.x, fma_(a.y, b.y, a.z * b.z)); }
template <class R>
__device__ __forceinline__ V3<R> cross(const V3<R>& a, const V3<R>& b) {
    return V3<R>{fma_(a.y, b.z, -(a.z * b.y)), fma_(a.z, b.x, -(a.x * b.z)), fma_(a.x, b.y, -(a.y * b.x))};
}
// s a + b
template <class R>
__device__ __forceinline__ V3<R> axpy(R s, const V3<R>& a, const V3<R>& b) {
    return V3<R>{fma_(s, a.x, b.x), fma_(s, a.y, b.y), fma_(s, a.z, b.z)};
}
template <class R>
__device__ __forceinline__ V3<R> operator+(const V3<R>& a, const V3<R>& b) { return V3<R>{a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R>
__device__ __forceinline__ V3<R> operator-(const V3<R>& a, const V3<R>& b) { return V3<R>{a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class R>
__device__ __forceinline__ V3<R> operator*(R s, const V3<R>& a) { return V3<R>{s * a.x, s * a.y, s * a.z}; }

// Division, reciprocal and square root.  FP64: IEEE operations.  FP32: the fixed approximate PTX
// instructions (relative error below 2^-22), written out so that the same source line rounds the same
// way at every inlining site (the FP32 translation units are built with IEEE division and square root
// and without contraction, so the compiler has no freedom left that could depend on the context).
__device__ __forceinline__ double rsqrt_(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsqrt_(float v) { return rsqrtf(v); }
__device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_(float v) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double rcp_(double v) { return 1.0 / v; }
__device__ __forceinline__ float rcp_(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
__device__ __forceinline__ float div_(float a, float b) { return a * rcp_(b); }
__device__ __forceinline__ double exp_(double v) { return exp(v); }
__device__ __forceinline__ float exp_(float v) { return expf(v); }
__device__ __forceinline__ void sincospi_(double v, double* s, double* c) { sincospi(v, s, c); }
__device__ __forceinline__ void sincospi_(float v, float* s, float* c) { sincospif(v, s, c); }
__device__ __forceinline__ double log_(double v) { return log(v); }
__device__ __forceinline__ float log_(float v) { return logf(v); }
__device__ __forceinline__ void sincos_(double v, double* s, double* c) { sincos(v, s, c); }
__device__ __forceinline__ void sincos_(float v, float* s, float* c) { sincosf(v, s, c); }

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t id, uint64_t seed, uint64_t step, uint32_t slot) {
    const uint64_t k = id ^ seed;
    return philox(make_uint4((uint32_t)step, (uint32_t)(step >> 32), slot, 0u), make_uint2((uint32_t)k, (uint32_t)(k >> 32)));
}

// 52 random bits -> (m + 1/2) 2^-52, exactly representable, strictly inside (0, 1).
__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
    const uint64_t m = ((uint64_t)(hi >> 12) << 32) | (uint64_t)lo;
    return ((double)m + 0.5) * 0x1.0p-52;
}

__device__ __forceinline__ double birth_tau(uint64_t id, uint64_t seed) {
    const uint4 w = draw(id, seed, kStepBirth, kSlotTauBranch);
    return -log(uniform52(w.x, w.y));
}

// ---------------------------------------------------------------------------------------------
// analytic plane-wave fields (stand-in for the grid fields of Sec. 4)
// ---------------------------------------------------------------------------------------------
template <class R>
struct FieldP {
    int kind;
    R a0, inv2n, phimax;  // envelope sin^2(phi * inv2n) on [0, phimax]
    R E0x, E0y, E0z, B0x, B0y, B0z;
    R eta0;
};

// sin and cos of a phase v + dv (dv a small correction): full precision in FP64; in FP32 v is reduced to
// [-pi, pi] with a two-term 2 pi (Cody-Waite), dv added there, and the hardware approximation evaluated
__device__ __forceinline__ void phase_sincos(double v, double* s, double* c, double dv = 0.0) { sincos(v + dv, s, c); }
__device__ __forceinline__ void phase_sincos(float v, float* s, float* c, float dv = 0.0f) {
    const float k = rintf(v * 0.15915494309189535f);
    const float r = fmaf(-k, 1.7484555e-07f, fmaf(-k, 6.28318548f, v)) + dv;  // 2 pi = 6.28318548 - 1.7484555e-7
    __sincosf(r, s, c);
}

// sin and cos of a phase v + dv to FP32 relative precision, zeros included (the event passes of the FP32
// path use it: there a field near a node enters chi and the photon energy relatively).  Quarter-period
// reduction with pi/2 split into three floats (Cody and Waite): P1 has 11 significant bits and P2 14, so
// k P1 and k P2 are exact for |k| < 2^10 (phases below ~1600 rad) and v - k P1 is exact; the remainder
// keeps its own relative precision down to the zeros of sin and cos.  For |r| <= pi/4 + |dv| the Taylor
// series of sin to r^11 and of cos to r^12 leave relative errors below 1e-11.
__device__ __forceinline__ void phase_sincos_acc(float v, float dv, float* s, float* c) {
    const float k = rintf(v * 0.636619772f);  // 2/pi
    float r = fmaf(-k, 1.5703125f, v);
    r = fmaf(-k, 4.838407039642334e-4f, r);
    r = fmaf(-k, -1.3909067675399456e-8f, r);
    r = r + dv;
    const float z = r * r;
    // sin r = r (1 - z/6 (1 - z/20 (1 - z/42 (1 - z/72 (1 - z/110))))), cos r likewise with 2, 12, ..., 132
    float ps = fmaf(-z, 1.0f / 110.0f, 1.0f);
    ps = fmaf(-z * (1.0f / 72.0f), ps, 1.0f);
    ps = fmaf(-z * (1.0f / 42.0f), ps, 1.0f);
    ps = fmaf(-z * (1.0f / 20.0f), ps, 1.0f);
    ps = fmaf(-z * (1.0f / 6.0f), ps, 1.0f);
    const float sr = r * ps;
    float pc = fmaf(-z, 1.0f / 132.0f, 1.0f);
    pc = fmaf(-z * (1.0f / 90.0f), pc, 1.0f);
    pc = fmaf(-z * (1.0f / 56.0f), pc, 1.0f);
    pc = fmaf(-z * (1.0f / 30.0f), pc, 1.0f);
    pc = fmaf(-z * (1.0f / 12.0f), pc, 1.0f);
    const float cr = fmaf(-z * 0.5f, pc, 1.0f);
    const int q = ((int)k) & 3;  // quadrant (two's complement: right for negative k too)
    const float sa = (q & 1) ? cr : sr, ca = (q & 1) ? sr : cr;
    *s = (q & 2) ? -sa : sa;
    *c = (q == 1 || q == 2) ? -ca : ca;
}
__device__ __forceinline__ void phase_sincos_acc(double v, double dv, double* s, double* c) { sincos(v + dv, s, c); }

// a + b as an unevaluated sum s + e (Knuth's TwoSum: e is the exact rounding error of s)
template <class R>
__device__ __forceinline__ R two_sum(R a, R b, R& e) {
    const R s = a + b;
    const R bp = s - a;
    e = (a - (s - bp)) + (b - bp);
    return s;
}

// (written as a select, not a branch: lanes of a warp straddle the pulse edges)
template <class R>
__device__ __forceinline__ R envelope(R phi, const FieldP<R>& f) {
    R s, c;
    phase_sincos(phi * f.inv2n, &s, &c);
    return (phi < R(0) || phi > f.phimax) ? R(0) : s * s;
}

// the envelope at the phase ps + dp to FP32 relative precision near its edges as well: the argument
// (ps + dp) inv2n as a product with its exact rounding error, then the accurate sine
template <class R>
__device__ __forceinline__ R envelope_acc(R ps, R dp, const FieldP<R>& f) {
    const R u = ps * f.inv2n;
    const R du = fma_(ps, f.inv2n, -u) + dp * f.inv2n;
    R s, c;
    phase_sincos_acc(u, du, &s, &c);
    const R phi = ps + dp;
    return (phi < R(0) || phi > f.phimax) ? R(0) : s * s;
}

// phase_t = t + phase (split by the caller for the FP32 path as hi + lo).  ACC: the accurate sine and
// cosine (event passes of the FP32 path); otherwise the fast ones.
// PW: the caller knows the field is a single plane wave (QED_FIELD_LP or QED_FIELD_CP)
template <class R, bool ACC = false, bool PW = false>
__device__ __forceinline__ void field_eval(const FieldP<R>& f, R ph_hi, R ph_lo, const V3<R>& x, V3<R>& E, V3<R>& B) {
    if (!PW && f.kind == QED_FIELD_CONST) {
        E = v3(f.E0x, f.E0y, f.E0z);
        B = v3(f.B0x, f.B0y, f.B0z);
        return;
    }
    if (!PW && f.kind == QED_FIELD_ROT_B) {  // |B| = B0z turning from z to y as t + phase runs over [0, phimax]
        R u = div_(ph_hi + ph_lo, f.phimax);
        u = u < R(0) ? R(0) : (u > R(1) ? R(1) : u);
        R sn, cs;
        sincospi_(R(0.5) * u, &sn, &cs);  // angle (pi/2) u, u in [0, 1]: no large-argument reduction
        E = v3(R(0), R(0), R(0));
        B = v3(R(0), f.B0z * sn, f.B0z * cs);
        return;
    }
    // phase t + phase - z: the rounding error of the subtraction is recovered exactly and added to the
    // reduced argument, so the FP32 carrier keeps the phase to ~1e-7 however large it is
    R e1;
    const R ps = two_sum(ph_hi, -x.z, e1);
    const R dp = e1 + ph_lo;
    const R phi = ps + dp;
    const R a = f.a0 * (ACC ? envelope_acc(ps, dp, f) : envelope(phi, f));
    E = v3(R(0), R(0), R(0));
    B = E;
    if (a != R(0)) {  // outside the envelope the carrier is not needed
        R s, c;
        if (ACC) phase_sincos_acc(ps, dp, &s, &c);
        else phase_sincos(ps, &s, &c, dp);
        const R ex = a * c, ey = f.kind == QED_FIELD_LP ? R(0) : a * s;
        E = v3(ex, ey, R(0));
        B = v3(-ey, ex, R(0));  // forward wave: B = z x E
    }
    if (!PW && f.kind == QED_FIELD_CP_COUNTER) {
        R e2;
        const R ps2 = two_sum(ph_hi, x.z, e2);
        const R dp2 = e2 + ph_lo;
        const R phi2 = ps2 + dp2;
        const R a2 = f.a0 * (ACC ? envelope_acc(ps2, dp2, f) : envelope(phi2, f));
        if (a2 != R(0)) {
            R s2, c2;
            if (ACC) phase_sincos_acc(ps2, dp2, &s2, &c2);
            else phase_sincos(ps2, &s2, &c2, dp2);
            const R ex2 = a2 * c2, ey2 = a2 * s2;
            E.x += ex2;
            E.y += ey2;
            B.x += ey2;  // backward wave: B = -z x E
            B.y += -ex2;
        }
    }
}

// The two waves of QED_FIELD_CP_COUNTER separately: the transverse E of the forward wave (B1 = z x E1) and
// of the backward wave (B2 = -z x E2), the same numbers field_eval adds up, so that a caller can form
// e E + p x B wave by wave.
template <class R>
struct Waves {
    R e1x, e1y, e2x, e2y;
};

template <class R, bool ACC = false>
__device__ __forceinline__ Waves<R> field_waves(const FieldP<R>& f, R ph_hi, R ph_lo, const V3<R>& x) {
    Waves<R> w{R(0), R(0), R(0), R(0)};
    R e1;
    const R ps = two_sum(ph_hi, -x.z, e1);
    const R dp = e1 + ph_lo;
    const R a = f.a0 * (ACC ? envelope_acc(ps, dp, f) : envelope(ps + dp, f));
    if (a != R(0)) {
        R s, c;
        if (ACC) phase_sincos_acc(ps, dp, &s, &c);
        else phase_sincos(ps, &s, &c, dp);
        w.e1x = a * c;
        w.e1y = a * s;
    }
    R e2;
    const R ps2 = two_sum(ph_hi, x.z, e2);
    const R dp2 = e2 + ph_lo;
    const R a2 = f.a0 * (ACC ? envelope_acc(ps2, dp2, f) : envelope(ps2 + dp2, f));
    if (a2 != R(0)) {
        R s2, c2;
        if (ACC) phase_sincos_acc(ps2, dp2, &s2, &c2);
        else phase_sincos(ps2, &s2, &c2, dp2);
        w.e2x = a2 * c2;
        w.e2y = a2 * s2;
    }
    return w;
}

// ---------------------------------------------------------------------------------------------
// classical pushers
// ---------------------------------------------------------------------------------------------
// Boris push of momentum p through dt with charge q (fields E, B).
template <class R>
__device__ __forceinline__ V3<R> boris(const V3<R>& p, const V3<R>& E, const V3<R>& B, R q, R dt) {
    const R h = R(0.5) * q * dt;
    const V3<R> pm = axpy(h, E, p);
    const R ig = rsqrt_(R(1) + dot(pm, pm));
    const V3<R> t = (h * ig) * B;
    const R sfac = div_(R(2), R(1) + dot(t, t));
    const V3<R> pp = pm + cross(pm, t);
    const V3<R> pl = pm + cross(pp, sfac * t);
    return axpy(h, E, pl);
}

// T-BMT precession vector Omega (ds/dt = Omega x s) with the time-centred momentum pb.
// ae: the anomalous moment (alpha/(2 pi), a(chi), or 0 for g = 2).
template <class R>
__device__ __forceinline__ V3<R> tbmt_omega(const V3<R>& pb, const V3<R>& E, const V3<R>& B, R q, bool paper_form, R ae) {
    const R gb = sqrt_(R(1) + dot(pb, pb));
    const R ig = rcp_(gb);
    const V3<R> bb = ig * pb;
    const R bB = dot(bb, B);
    const V3<R> bxE = cross(bb, E);
    const R c1 = ae + ig, c2 = div_(ae * gb, gb + R(1));
    if (paper_form)  // (a + 1/gamma)(B - v x E) - (a gamma/(gamma+1))(v.B) v, as printed in Sec. 8.3
        return (-q) * axpy(-(c2 * bB), bb, c1 * (B - bxE));
    // standard form: (a + 1/gamma) B - (a gamma/(gamma+1))(beta.B) beta - (a + 1/(gamma+1)) beta x E
    const R c3 = ae + rcp_(gb + R(1));
    return (-q) * axpy(-c3, bxE, axpy(-(c2 * bB), bb, c1 * B));
}

// rotate s about Omega by |Omega| dt (Rodrigues)
template <class R>
__device__ __forceinline__ V3<R> rotate(const V3<R>& s, const V3<R>& Om, R dt) {
    const R o2 = dot(Om, Om);
    if (!(o2 > R(0))) return s;
    const R io = rsqrt_(o2);
    const V3<R> n = io * Om;
    R sn, c;
    phase_sincos(o2 * io * dt, &sn, &c);
    const V3<R> nxs = cross(n, s);
    const R ns = dot(n, s);
    return axpy(ns * (R(1) - c), n, axpy(sn, nxs, c * s));
}

// chi = eta0 sqrt((e E + p x B)^2 - (p.E)^2)
template <class R>
__device__ __forceinline__ R chi_of(R eta0, R e, const V3<R>& p, const V3<R>& E, const V3<R>& B) {
    const V3<R> a = axpy(e, E, cross(p, B));
    const R pe = dot(p, E);
    const R v = fma_(-pe, pe, dot(a, a));
    return eta0 * sqrt_(v > R(0) ? v : R(0));
}

// (eps, beta): eps along the part of f = E + v x B perpendicular to khat, times `sign`;
// beta = khat x eps (right-handed basis).  Returns false if undefined.
template <class R>
__device__ __forceinline__ bool make_basis(const V3<R>& E, const V3<R>& B, const V3<R>& v, const V3<R>& khat, R sign,
                                           V3<R>& eps, V3<R>& beta) {
    const V3<R> f = E + cross(v, B);
    const R fk = dot(f, khat);
    const V3<R> fp = axpy(-fk, khat, f);
    const R n2 = dot(fp, fp);
    if (!(n2 > R(0))) return false;
    eps = (sign * rsqrt_(n2)) * fp;
    beta = cross(khat, eps);
    return true;
}

// ---------------------------------------------------------------------------------------------
// spectra of App. A (Bessel forms); bes = (K13, K23, IntK13) at the event's u' (any common scale)
// ---------------------------------------------------------------------------------------------
// NLC: w = -IntK13 + kappa K23 + lambda (s_i.beta) K13 ;
//      g = u K13 beta + (-IntK13 + 2 K23) s_i + lambda u (-IntK13 + K23)(s_i.k) k
template <class R>
__device__ __forceinline__ void nlc_wg(R lam, R one_m, const R bes[3], const V3<R>& si, const V3<R>& beta,
                                       const V3<R>& k, R& w, V3<R>& g) {
    const R u = div_(lam, one_m);
    const R kappa = rcp_(one_m) + one_m;
    const R K13 = bes[0], K23 = bes[1], IK = bes[2];
    w = -IK + kappa * K23 + lam * dot(si, beta) * K13;
    g = (u * K13) * beta + (-IK + R(2) * K23) * si + (lam * u * (-IK + K23) * dot(si, k)) * k;
}

// NLC photon Stokes spectrum F = (F0, F1, F2, F3), App. A.1 Eqs. F0-F3.
template <class R>
__device__ __forceinline__ void nlc_stokes(R lam, R one_m, const R bes[3], const V3<R>& si, const V3<R>& sf, R w,
                                           const V3<R>& g, const V3<R>& eps, const V3<R>& beta, const V3<R>& k,
                                           R F[4]) {
    const R u = div_(lam, one_m);
    const R kappa = rcp_(one_m) + one_m;
    const R kappat = rcp_(one_m) - one_m;
    const R K13 = bes[0], K23 = bes[1], IK = bes[2];
    const R sie = dot(si, eps), sib = dot(si, beta), sik = dot(si, k);
    const R sfe = dot(sf, eps), sfb = dot(sf, beta), sfk = dot(sf, k);
    const V3<R> fxi = cross(sf, si);
    const R lu2 = R(0.5) * lam * u;
    F[0] = w + dot(sf, g);
    F[1] = -K13 * (u * sie + lam * sfe) - lu2 * IK * (sfe * sib + sfb * sie) + R(0.5) * kappat * K23 * dot(fxi, k);
    F[2] = R(0.5) * kappat * K13 * dot(fxi, eps) - (lam * IK - kappat * K23) * sik - (u * IK - kappat * K23) * sfk +
           lu2 * K13 * (sfk * sib + sfb * sik);
    F[3] = K23 + (u * sib + lam * sfb) * K13 - lu2 * IK * (sfe * sie - sfb * sib) + R(0.5) * kappa * K23 * dot(sf, si) -
           lu2 * K23 * sfk * sik;
}

// NBW expected daughter spins (App. A.2): w0, j_e, j_p for positron fraction lam.
template <class R>
__device__ __forceinline__ void nbw_j(R lam, R one_m, const R bes[3], const R xi[3], const V3<R>& eps, const V3<R>& beta,
                                      const V3<R>& k, R& w0, V3<R>& je, V3<R>& jp) {
    const R il = rcp_(lam), im = rcp_(one_m);
    const R rho = one_m * il + lam * im;
    const R rhot = one_m * il - lam * im;
    const R K13 = bes[0], K23 = bes[1], IK = bes[2];
    w0 = IK + rho * K23 - xi[2] * K23;
    je = ((im - xi[2] * il) * K13) * beta + (xi[0] * il * K13) * eps + (xi[1] * (im * IK + rhot * K23)) * k;
    jp = ((-il + xi[2] * im) * K13) * beta + (-xi[0] * im * K13) * eps + (xi[1] * (il * IK - rhot * K23)) * k;
}

// NBW full spectrum contracted with xi: G0 + xi . (G1, G2, G3) (App. A.2 Eqs. G0-G3; the last term of G3
// with the sign of its Airy form).
template <class R>
__device__ __forceinline__ R nbw_G(R lam, R one_m, const R bes[3], const R xi[3], const V3<R>& sp, const V3<R>& se,
                                   const V3<R>& eps, const V3<R>& beta, const V3<R>& k) {
    const R il = rcp_(lam), im = rcp_(one_m);
    const R rho = one_m * il + lam * im;
    const R rhot = one_m * il - lam * im;
    const R ut = il + im;
    const R K13 = bes[0], K23 = bes[1], IK = bes[2];
    const R spe = dot(sp, eps), spb = dot(sp, beta), spk = dot(sp, k);
    const R see = dot(se, eps), seb = dot(se, beta), sek = dot(se, k);
    const V3<R> pxe = cross(sp, se);
    const R sps = dot(sp, se);
    const R G0 = IK + rho * K23 + im * seb * K13 - il * spb * K13 + (IK - R(2) * K23) * sps +
                 (rho * IK - (rho - R(2)) * K23) * spk * sek;
    const R G1 = K13 * (il * see - im * spe) - R(0.5) * ut * IK * (spe * seb + spb * see) + R(0.5) * rhot * K23 * dot(pxe, k);
    const R G2 = -R(0.5) * ut * K13 * dot(pxe, eps) + (im * IK + rhot * K23) * sek + (il * IK - rhot * K23) * spk -
                 R(0.5) * rhot * K13 * (spk * seb + spb * sek);
    const R G3 = -K23 + (-il * seb + im * spb) * K13 - R(0.5) * ut * IK * (spe * see - spb * seb) + R(0.5) * rho * K23 * sps +
                 (R(1) - R(0.5) * rho) * K23 * spk * sek;
    return G0 + xi[0] * G1 + xi[1] * G2 + xi[2] * G3;
}

// Stokes -> P (Sec. 3.2): P = xi2 k + l (cos dth eps + sin dth beta), l = |(xi1, xi3)|, 2 dth = atan2(xi1, xi3),
// with half-angle identities: (l cos dth)^2 = l (l + xi3)/2, (l sin dth)^2 = l (l - xi3)/2 and
// (l cos dth)(l sin dth) = l xi1 / 2.  The larger component comes from its square root (no cancellation),
// the smaller one from the product; cos dth >= 0.
// Both cases are evaluated with the same operations and chosen by selects (no divergent branch).
template <class R>
__device__ __forceinline__ V3<R> stokes_to_P(const R xi[3], const V3<R>& eps, const V3<R>& beta, const V3<R>& k) {
    const R l = sqrt_(xi[0] * xi[0] + xi[2] * xi[2]);
    const bool up = xi[2] >= R(0);  // cos dth is the larger component
    const R half = R(0.5) * l * xi[0];
    R big = sqrt_(R(0.5) * l * (up ? l + xi[2] : l - xi[2]));
    if (!up && xi[0] < R(0)) big = -big;
    const R small = div_(half, big);
    const bool some = l > R(0);
    const R c = some ? (up ? big : small) : R(0);
    const R s = some ? (up ? small : big) : R(0);
    return axpy(s, beta, axpy(c, eps, xi[1] * k));
}

// P -> Stokes in the basis (eps, beta, k): xi1 = 2 P1 P2 / l, xi2 = P.k, xi3 = (P1^2 - P2^2)/l.
template <class R>
__device__ __forceinline__ void P_to_stokes(const V3<R>& P, const V3<R>& eps, const V3<R>& beta, const V3<R>& k, R xi[3]) {
    const R P1 = dot(P, eps), P2 = dot(P, beta);
    const R l2 = P1 * P1 + P2 * P2;
    xi[1] = dot(P, k);
    const bool some = l2 > R(0);
    const R il = rsqrt_(some ? l2 : R(1));
    xi[0] = some ? R(2) * P1 * P2 * il : R(0);
    xi[2] = some ? (P1 * P1 - P2 * P2) * il : R(0);
}

// ---------------------------------------------------------------------------------------------
// block-level counter reduction: one atomic per block and counter
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int N>
__device__ __forceinline__ void flush_counters(unsigned long long (&c)[N], unsigned long long* dst) {
    __shared__ unsigned long long red[32][N];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) c[i] = warp_sum(c[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[wid][i] = c[i];
    __syncthreads();
    if (threadIdx.x < N) {
        unsigned long long s = 0;
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
        if (s) atomicAdd(dst + threadIdx.x, s);
    }
}

// The first error wins.  Once the status is set (the common case when a buffer overflows on every
// event of a step) a plain load sees it and no atomic is issued, so a flood of errors does not
// serialise on the one word.
__device__ __forceinline__ void record_error(qed_counters* ctr, int32_t status, int64_t idx) {
    if (*reinterpret_cast<volatile int32_t*>(&ctr->status) != 0) return;
    if (atomicCAS(&ctr->status, 0, status) == 0) ctr->first_bad = idx;
}

// ---------------------------------------------------------------------------------------------
// budgeted daughter appends
// ---------------------------------------------------------------------------------------------
// The daughter buffers of one step call (or of one instance's step in a batch) take the counts they had
// when the step began (base), how many events' daughters fit (budget) and how many events asked (next).
// Event k of the call (k in reservation order) writes its daughters at base + k if k < budget, else it
// is not applied; afterwards each count becomes base + min(next, budget).  A pair therefore goes into
// both buffers or into neither, and no count ever exceeds its capacity.  The layout matches the
// append_* fields at the end of qed_counters.
struct AppendState {
    int64_t base[2];   // the daughter buffers' counts when the step began (pairs: electrons, positrons)
    int64_t budget;    // events whose daughters fit
    unsigned long long next;  // events that asked for slots
};

// open the reservation of a step: c1 may be NULL (one daughter buffer)
__device__ __forceinline__ void append_open(AppendState* A, const int64_t* c0, int64_t cap0, const int64_t* c1,
                                            int64_t cap1) {
    const int64_t n0 = min(max(*c0, (int64_t)0), cap0);
    int64_t budget = cap0 - n0;
    A->base[0] = n0;
    A->base[1] = 0;
    if (c1) {
        const int64_t n1 = min(max(*c1, (int64_t)0), cap1);
        A->base[1] = n1;
        budget = min(budget, cap1 - n1);
    }
    A->budget = budget;
    A->next = 0ull;
}

// close it: the counts after the step's appends
__device__ __forceinline__ void append_close(const AppendState* A, int64_t* c0, int64_t* c1) {
    const int64_t used = min((int64_t)A->next, A->budget);
    *c0 = A->base[0] + used;
    if (c1) *c1 = A->base[1] + used;
}

// Event index of this lane in its reservation (all 32 lanes call it; lanes may name different states:
// the lanes of one state form a group whose first wanting lane reserves for the group with one atomic
// add).  -1 for lanes that do not want a slot or name no state; otherwise the caller compares the index
// with the budget.
__device__ __forceinline__ long long reserve_event(AppendState* A, bool want) {
    want = want && A != nullptr;
    const unsigned grp = __match_any_sync(0xffffffffu, (unsigned long long)A);
    const unsigned m = __ballot_sync(0xffffffffu, want) & grp;
    if (m == 0) return -1;  // uniform over the group
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    long long base = 0;
    if (lane == leader) base = (long long)atomicAdd(&A->next, (unsigned long long)__popc(m));
    base = __shfl_sync(grp, base, leader);
    return want ? base + (long long)__popc(m & ((1u << lane) - 1u)) : -1;
}

// warp-aggregated slot reservation on a device counter: returns the slot of this lane (valid if want)
__device__ __forceinline__ long long reserve_slots(int64_t* counter, bool want, int per) {
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    if (mask == 0) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    long long base = 0;
    if (lane == leader) base = (long long)atomicAdd((unsigned long long*)counter, (unsigned long long)(__popc(mask) * per));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + (long long)(__popc(mask & ((1u << lane) - 1u)) * per);
}

}  // namespace qed
