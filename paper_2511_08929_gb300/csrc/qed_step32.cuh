// qed_step32.cuh -- the per-particle arithmetic of the FP32 fast path, shared by the single-buffer step
// kernels (qed_step32.cu) and the batched persistent kernel (qed_batch.cu).
//
// Arithmetic split (Sec. 5.1, 5.2, 6): the Boris and T-BMT pushers, chi, the basis, the rate lookups and
// all event sampling in FP32; the optical depth is accumulated in FP64 and the excess |s|^2 - 1 of a
// spin / Stokes vector that leaves the unit ball is computed in FP64.  Particles are three float4 planes:
// leptons q0 = (x, y, z, p_x), q1 = (p_y, p_z, s_x, s_y), q2 = (s_z, w, tau_lo, tau_hi); photons
// q0 = (x, y, z, P_x), q1 = (P_y, P_z, tau_lo, tau_hi), q2 = (k_x, k_y, k_z, w), so that a photon step,
// which never changes k or w, writes two planes (one when the photon has no pair rate).
#pragma once
#include "qed_bessel.cuh"
#include "qed_internal.h"
#include "qed_steps.h"

// How the event passes (lepton_events, photon_events) are compiled into their caller: out of line in
// the single-buffer kernels, whose streaming loop stays free of their registers; the batched event
// kernel, which runs nothing else, defines it as __forceinline__ (one block of 256 threads per SM then
// holds the whole pass in registers without the call frames' local-memory traffic).
#ifndef QED_EVENT_PASS
#define QED_EVENT_PASS __noinline__
#endif

namespace qed {

using F3 = V3<float>;
constexpr int kT32 = 256;  // threads per block
constexpr int kWarps32 = kT32 / 32;
constexpr int kStages = 3;  // tiles in flight per warp
constexpr int kWQ = 64;     // queued event indices per warp (drained 32 at a time)
constexpr int kWaitLimit = 1 << 24;  // bounded mbarrier polling (~0.1 s) before reporting a timeout

struct Tile {  // one tile of 32 particles in shared memory
    float4 q0[32], q1[32], q2[32];
};

// ------------------------------------------------------------------------------------------------
// bulk copies and mbarriers (PTX)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of `parity` to complete (false: gave up)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < kWaitLimit; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------------------------------------------
// numeric helpers
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double tau_join(float lo, float hi) { return __hiloint2double(__float_as_int(hi), __float_as_int(lo)); }
__device__ __forceinline__ void tau_split(double t, float& lo, float& hi) {
    lo = __int_as_float(__double2loint(t));
    hi = __int_as_float(__double2hiint(t));
}

// FP32 uniforms from the Philox words.  The method's uniform is u = (m + 1/2) 2^-52 with the 52-bit
// m = (hi >> 12) 2^32 + lo (exactly as in the FP64 path); here it is rounded to float with two 32-bit
// integer conversions, and 1 - u is formed from the complementary integer 2^52 - 1 - m, so neither
// end of (0, 1) loses precision.
__device__ __forceinline__ float u52f_parts(uint32_t h20, uint32_t lo) {
    return fmaf((float)h20, 0x1.0p-20f, ((float)lo + 0.5f) * 0x1.0p-52f);
}
__device__ __forceinline__ float u52f(uint32_t hi, uint32_t lo) { return u52f_parts(hi >> 12, lo); }
__device__ __forceinline__ float u52f_comp(uint32_t hi, uint32_t lo) { return u52f_parts(0xFFFFFu - (hi >> 12), ~lo); }

// logit ln(u) - ln(1 - u) of the uniform (full-accuracy logf: it is the ICDF coordinate)
__device__ __forceinline__ float logit52(uint32_t hi, uint32_t lo) { return logf(u52f(hi, lo)) - logf(u52f_comp(hi, lo)); }

// exponential draw -ln(u) (an optical depth), sampled in FP32 and widened to the FP64 accumulator
__device__ __forceinline__ double exp_draw(uint32_t hi, uint32_t lo) {
    const float u = u52f(hi, lo);
    return (double)(u < 0.5f ? -logf(u) : -log1pf(-u52f_comp(hi, lo)));
}

__device__ __forceinline__ double birth_tau32(uint64_t id, uint64_t seed) {
    const uint4 w = draw(id, seed, kStepBirth, kSlotTauBranch);
    return exp_draw(w.x, w.y);
}

// A positive normal float widened to double exactly by rearranging its bits on the integer units (the
// FP64 pipe of this GPU is narrow): sign 0, exponent rebased from 127 to 1023, mantissa moved up 29
// bits.  Zero, denormals, negatives, infinities and NaNs take the plain conversion.
__device__ __forceinline__ double widen_pos(float v) {
    const uint32_t u = __float_as_uint(v);
    if (u < 0x00800000u || u >= 0x7F800000u) return (double)v;
    const uint32_t hi = (((u >> 23) + (1023u - 127u)) << 20) | ((u & 0x7FFFFFu) >> 3);
    const uint32_t lo = u << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// A spin or Stokes vector is renormalised when |s|^2 exceeds 1 by more than the FP32 rounding of the
// update that produced it; below that the excess is rounding noise (the exact update of Sec. 6 raises
// |s|^2 by (P dt)^2 (1 - (s.beta)^2) / D^2, a real second-order excess, which still triggers it).
constexpr float kRenormSlack = 0x1.0p-20f;

// Rescale a vector that left the unit ball.  Its excess d = |s|^2 - 1 is computed in FP64 (the
// products of floats are exact in double, so d is exact to 1e-16); the factor (1 + d)^{-1/2} =
// 1 - d/2 + 3 d^2/8 (relative error 5 d^3/16 < 1e-11 for d < 2^-10) is then applied in FP32, whose
// rounding is the precision of the stored state.  Larger excursions take the FP32 reciprocal root.
__device__ __forceinline__ F3 renorm64(const F3& s) {
    const double x = s.x, y = s.y, z = s.z;
    const double d = fma(x, x, fma(y, y, fma(z, z, -1.0)));
    const float df = (float)d;
    float f;
    if (df < 0x1.0p-10f) {
        f = fmaf(df, fmaf(0.375f, df, -0.5f), 1.0f);
    } else {
        const float n2 = 1.0f + df;
        f = rsqrtf(n2);
        f = f * (1.5f - 0.5f * n2 * f * f);
    }
    return F3{s.x * f, s.y * f, s.z * f};
}

// optical depth decision tau <= 0 as an integer test on the FP64 bit pattern (+0 and every value
// with the sign bit set compare <= 0 as signed 64-bit integers)
__device__ __forceinline__ bool tau_spent(double t) { return __double_as_longlong(t) <= 0ll; }

// true if the ten state words a particle's step reads (x, p or k, s or P, w) are all finite: 0 * v is
// zero for finite v and NaN for infinities and NaNs, so the fused sum below is zero exactly when all are
__device__ __forceinline__ bool finite_state(const float4& a, const float4& b, const float4& cc) {
    float z = 0.0f * a.x;
    z = fmaf(0.0f, a.y, z);
    z = fmaf(0.0f, a.z, z);
    z = fmaf(0.0f, a.w, z);
    z = fmaf(0.0f, b.x, z);
    z = fmaf(0.0f, b.y, z);
    z = fmaf(0.0f, b.z, z);
    z = fmaf(0.0f, b.w, z);
    z = fmaf(0.0f, cc.x, z);
    z = fmaf(0.0f, cc.y, z);
    return z == 0.0f;
}

// the same test for a photon's planes: x and P_x (q0), P_y and P_z (q1), k and w (q2)
__device__ __forceinline__ bool finite_photon(const float4& a, const float4& b, const float4& cc) {
    float z = 0.0f * a.x;
    z = fmaf(0.0f, a.y, z);
    z = fmaf(0.0f, a.z, z);
    z = fmaf(0.0f, a.w, z);
    z = fmaf(0.0f, b.x, z);
    z = fmaf(0.0f, b.y, z);
    z = fmaf(0.0f, cc.x, z);
    z = fmaf(0.0f, cc.y, z);
    z = fmaf(0.0f, cc.z, z);
    z = fmaf(0.0f, cc.w, z);
    return z == 0.0f;
}

// ------------------------------------------------------------------------------------------------
// shared memory
// ------------------------------------------------------------------------------------------------
struct Shared32 {
    float* bes;      // [3][kBesN]
    float* rates;    // nlc [2][n_chi] then nbw [2][n_chi]
    Tile* tiles;     // [warps][kStages]
    uint64_t* bars;  // [warps][kStages]
    int64_t* queue;  // [warps][kWQ]
};

__host__ __device__ inline size_t align128(size_t b) { return (b + 127) & ~size_t(127); }

__host__ __device__ inline size_t smem32_bytes(int n_chi) {
    return align128((size_t)3 * kBesN * 4 + (size_t)4 * n_chi * 4) + (size_t)kWarps32 * kStages * sizeof(Tile) +
           (size_t)kWarps32 * kStages * 8 + (size_t)kWarps32 * kWQ * 8;
}

__device__ __forceinline__ Shared32 carve32(unsigned char* smem, int n_chi) {
    Shared32 s;
    s.bes = (float*)smem;
    s.rates = s.bes + 3 * kBesN;
    size_t off = align128((size_t)3 * kBesN * 4 + (size_t)4 * n_chi * 4);
    s.tiles = (Tile*)(smem + off);
    off += (size_t)kWarps32 * kStages * sizeof(Tile);
    s.bars = (uint64_t*)(smem + off);
    off += (size_t)kWarps32 * kStages * 8;
    s.queue = (int64_t*)(smem + off);
    return s;
}

__device__ __forceinline__ void load_tables32(const Shared32& sh, const float* __restrict__ bes_g, const TabP<float>& T) {
    for (int i = threadIdx.x; i < 3 * kBesN; i += blockDim.x) sh.bes[i] = bes_g[i];
    for (int i = threadIdx.x; i < 2 * T.n_chi; i += blockDim.x) {
        sh.rates[i] = T.nlc_rate[i];
        sh.rates[2 * T.n_chi + i] = T.nbw_rate[i];
    }
}

enum { C_EVENTS, C_STORED, C_DROPPED, C_CLAMPED, C_RENORM, C_BELOW, C_NONFINITE, C_RATE_STEPS, C_BOUND, C_N };

// per-warp counter flush (no block barrier: warps finish at different times)
__device__ __forceinline__ void flush_warp(unsigned long long (&c)[C_N], qed_counters* ctr) {
#pragma unroll
    for (int i = 0; i < C_N; ++i) {
        const unsigned long long v = warp_sum(c[i]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&ctr->events + i, v);
    }
}

// The warp's tile stream: tile t of this warp covers particles [32 g_t, 32 g_t + 32), g_t = g_0 + t G.
struct TileStream {
    Tile* tile;      // this warp's kStages tiles
    uint64_t* bar;   // this warp's kStages mbarriers
    const float4 *q0, *q1, *q2;
    int64_t n, g0, G;

    __device__ __forceinline__ int64_t base(int64_t t) const { return (g0 + t * G) * 32; }
    // lane 0: start the copies of tile t into stage t % kStages
    __device__ __forceinline__ void issue(int64_t t) const {
        const int64_t b = base(t);
        if (b >= n) return;
        const int s = (int)(t % kStages);
        const uint32_t bytes = (uint32_t)(min((int64_t)32, n - b) * 16);
        mbar_expect_tx(&bar[s], 3 * bytes);
        bulk_g2s(tile[s].q0, q0 + b, bytes, &bar[s]);
        bulk_g2s(tile[s].q1, q1 + b, bytes, &bar[s]);
        bulk_g2s(tile[s].q2, q2 + b, bytes, &bar[s]);
    }
};

// Slot reservation on per-lane device counters (all 32 lanes call it): the lanes that name the same
// counter form one group, whose first wanting lane takes the group's slots with one atomic add; a lane
// that does not want a slot (or names no counter) gets -1.  Lanes of one event pass may belong to
// different buffers (the batched event kernel takes events of several instances at once).
__device__ __forceinline__ long long reserve_grouped(int64_t* counter, bool want) {
    want = want && counter != nullptr;
    const unsigned grp = __match_any_sync(0xffffffffu, (unsigned long long)counter);
    const unsigned m = __ballot_sync(0xffffffffu, want) & grp;
    if (m == 0) return -1;  // uniform over the group
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    long long base = 0;
    if (lane == leader) base = (long long)atomicAdd((unsigned long long*)counter, (unsigned long long)__popc(m));
    base = __shfl_sync(grp, base, leader);
    return want ? base + (long long)__popc(m & ((1u << lane) - 1u)) : -1;
}

// ------------------------------------------------------------------------------------------------
// lepton step
// ------------------------------------------------------------------------------------------------
struct Ctx {
    TabP<float> T;  // rates point to shared memory, ICDFs to global
    const float* bes;
    FieldP<float> F;
    StepP S;
    float q;
};

// the step flags: FIX when the caller fixes them at compile time (nonzero), else the context's
template <uint32_t FIX>
__device__ __forceinline__ uint32_t flags_of(const Ctx& C) {
    return FIX ? FIX : C.S.flags;
}

// chi and the basis vector f = E + v x B for the FP32 path, in forms free of the cancellation that the
// general ones suffer for a particle moving with a wave (there e E and p x B nearly cancel, and the
// general forms lose ~1/theta^2 of relative precision at an angle theta to the wave).  With
// e - p_z and e + p_z from e_minus_pz / e_plus_pz (no difference of nearly equal numbers):
//   a single wave along +z (the linear and circular lasers; E transverse, B = z x E):
//     chi = eta0 (e - p_z) |E|,   f = ((e - p_z) E + (p.E) z) / e;
//   the counter-propagating pair (E1 forward with B1 = z x E1, E2 backward with B2 = -z x E2):
//     chi^2 = eta0^2 (|(e - p_z) E1 + (e + p_z) E2|^2 - 4 (p.E1)(p.E2)),
//     f = ((e - p_z) E1 + (e + p_z) E2 + (p.E1 - p.E2) z) / e;
// both are e E + p x B and the invariant chi^2 = eta0^2 ((e E + p x B)^2 - (p.E)^2) written out for
// these fields.  Other fields take the general forms.
__device__ __forceinline__ bool single_wave(const Ctx& C) {
    return C.F.kind == QED_FIELD_LP || C.F.kind == QED_FIELD_CP;
}

__device__ __forceinline__ bool two_wave(const Ctx& C) { return C.F.kind == QED_FIELD_CP_COUNTER; }

// The batched kernels built for a fixed flag set (FIX != 0) run only batches whose instances are all
// single plane waves (the linear and circular lasers); the host picks them so.  They carry no code for
// the other field kinds.
template <uint32_t FIX>
__device__ __forceinline__ constexpr bool plane_waves_only() {
    return FIX != 0;
}

// e - p_z of a particle with e^2 = m2 + p^2 (m2 = 1 lepton, 0 photon): where it moves with the forward
// wave (p_z > 0) e and p_z nearly cancel, and it is taken as (m2 + p_x^2 + p_y^2) / (e + p_z)
__device__ __forceinline__ float e_minus_pz(float e, const F3& p, float m2) {
    return p.z > 0.0f ? div_(fma_(p.x, p.x, fma_(p.y, p.y, m2)), e + p.z) : e - p.z;
}

// chi and f = E + v x B of the counter-propagating pair from its two waves (the forms above)
struct ChiF {
    float chi;
    F3 f;
};

__device__ __forceinline__ ChiF two_wave_chi(const Waves<float>& w, float eta0, float e, const F3& p, float m2) {
    const float q = fma_(p.x, p.x, fma_(p.y, p.y, m2));
    float em, ep;
    if (p.z > 0.0f) {
        ep = e + p.z;
        em = div_(q, ep);
    } else {
        em = e - p.z;
        ep = div_(q, em);
    }
    const float tx = fma_(em, w.e1x, ep * w.e2x), ty = fma_(em, w.e1y, ep * w.e2y);
    const float pe1 = fma_(p.x, w.e1x, p.y * w.e1y), pe2 = fma_(p.x, w.e2x, p.y * w.e2y);
    const float ie = rcp_(e);
    const float v = fma_(-4.0f * pe1, pe2, fma_(tx, tx, ty * ty));
    return ChiF{eta0 * sqrt_(v > 0.0f ? v : 0.0f), F3{ie * tx, ie * ty, ie * (pe1 - pe2)}};
}

// xold: where the fields were evaluated (the counter-propagating field is evaluated again there, wave by
// wave); the result's f is set for that kind only (basis32 takes it from there)
template <bool ACC, bool PW>
__device__ __forceinline__ ChiF chi32(const Ctx& C, float e, const F3& p, const F3& E, const F3& B, float m2,
                                     const F3& xold) {
    if (PW || single_wave(C)) return ChiF{C.F.eta0 * e_minus_pz(e, p, m2) * sqrt_(fma_(E.x, E.x, E.y * E.y)), F3{0, 0, 0}};
    if (two_wave(C))
        return two_wave_chi(field_waves<float, ACC>(C.F, C.S.ph_hi_f, C.S.ph_lo_f, xold), C.F.eta0, e, p, m2);
    return ChiF{chi_of(C.F.eta0, e, p, E, B), F3{0, 0, 0}};
}

// ie = 1/e; f2w: f of the counter-propagating field from chi32
template <bool PW>
__device__ __forceinline__ bool basis32(const Ctx& C, const F3& E, const F3& B, const F3& v, const F3& khat, float sign,
                                       F3& eps, F3& beta, float ie, const F3& p, float m2, const F3& f2w) {
    F3 f;
    if (PW || single_wave(C)) {
        const float g = e_minus_pz(1.0f / ie, p, m2) * ie;
        f = F3{g * E.x, g * E.y, fma_(v.x, E.x, v.y * E.y)};
    } else if (two_wave(C)) {
        f = f2w;
    } else {
        f = E + cross(v, B);
    }
    const float fk = dot(f, khat);
    const F3 fp = axpy(-fk, khat, f);
    const float n2 = dot(fp, fp);
    if (!(n2 > 0.0f)) return false;
    eps = (sign * rsqrtf(n2)) * fp;
    beta = cross(khat, eps);
    return true;
}

// The Boris push and the T-BMT vector for fields with E_z = B_z = 0 (the plane waves along z: the
// linear, circular and counter-propagating circular lasers): the general forms with the products by the
// zero components left out.  A product by zero only adds a signed zero, so for finite inputs the results
// equal the general forms' up to the sign of a zero result.
__device__ __forceinline__ F3 cross_t(const F3& a, const F3& b) {  // b.z = 0
    return F3{-(a.z * b.y), a.z * b.x, fma_(a.x, b.y, -(a.y * b.x))};
}

// The Boris rotation of p- by t = (q dt/2) B / gamma- in closed form,
//   p+ = c p- + s (p- x t) + s (t.p-) t,   s = 2/(1 + t^2), c = s - 1 = (1 - t^2)/(1 + t^2),
// which is the textbook p+ = p- + (p- + p- x t) x s t written out: every term is bounded by |p-|
// (2|t|/(1 + t^2) <= 1), so the FP32 rounding stays at a few ulp of |p| where a step turns the momentum by
// a large angle (|t| >> 1: low-energy leptons in strong fields), where the textbook form's intermediate
// p- x t is |t| times larger than the result.  pb receives the time-centred momentum (p_old + p_new)/2 =
// (p- + p+)/2 = (s/2)(p- + p- x t + (t.p-) t), free of the cancellation of the average of two momenta a
// large turn apart.
__device__ __forceinline__ F3 boris_t(const F3& p, const F3& E, const F3& B, float q, float dt, F3& pb) {
    const float h = 0.5f * q * dt;
    const F3 pm{fma_(h, E.x, p.x), fma_(h, E.y, p.y), p.z};
    const float ig = rsqrt_(1.0f + dot(pm, pm));
    const float hi = h * ig;
    const F3 t{hi * B.x, hi * B.y, 0.0f};
    const float sf = div_(2.0f, 1.0f + fma_(t.x, t.x, t.y * t.y));
    const float c = sf - 1.0f, stp = sf * fma_(t.x, pm.x, t.y * pm.y);
    const F3 x = cross_t(pm, t);
    const F3 pl{fma_(c, pm.x, fma_(sf, x.x, stp * t.x)), fma_(c, pm.y, fma_(sf, x.y, stp * t.y)), fma_(c, pm.z, sf * x.z)};
    const float hs = 0.5f * sf, hstp = 0.5f * stp;
    pb = F3{fma_(hs, pm.x + x.x, hstp * t.x), fma_(hs, pm.y + x.y, hstp * t.y), hs * (pm.z + x.z)};
    return F3{fma_(h, E.x, pl.x), fma_(h, E.y, pl.y), pl.z};
}

// the same for fields with E_z or B_z nonzero
__device__ __forceinline__ F3 boris32(const F3& p, const F3& E, const F3& B, float q, float dt, F3& pb) {
    const float h = 0.5f * q * dt;
    const F3 pm = axpy(h, E, p);
    const float ig = rsqrt_(1.0f + dot(pm, pm));
    const F3 t = (h * ig) * B;
    const float sf = div_(2.0f, 1.0f + dot(t, t));
    const float c = sf - 1.0f, stp = sf * dot(t, pm);
    const F3 x = cross(pm, t);
    const F3 pl{fma_(c, pm.x, fma_(sf, x.x, stp * t.x)), fma_(c, pm.y, fma_(sf, x.y, stp * t.y)),
                fma_(c, pm.z, fma_(sf, x.z, stp * t.z))};
    const float hs = 0.5f * sf, hstp = 0.5f * stp;
    pb = F3{fma_(hs, pm.x + x.x, hstp * t.x), fma_(hs, pm.y + x.y, hstp * t.y), fma_(hs, pm.z + x.z, hstp * t.z)};
    return axpy(h, E, pl);
}

__device__ __forceinline__ F3 tbmt_omega_t(const F3& pb, const F3& E, const F3& B, float q, bool paper_form, float ae) {
    const float gb = sqrt_(1.0f + dot(pb, pb));
    const float ig = rcp_(gb);
    const F3 bb = ig * pb;
    const float bB = fma_(bb.x, B.x, bb.y * B.y);
    const F3 bxE = cross_t(bb, E);
    const float c1 = ae + ig, c2 = div_(ae * gb, gb + 1.0f);
    if (paper_form) return (-q) * axpy(-(c2 * bB), bb, c1 * F3{B.x - bxE.x, B.y - bxE.y, 0.0f - bxE.z});
    const float c3 = ae + rcp_(gb + 1.0f);
    const float m = -(c2 * bB);
    const F3 w{fma_(m, bb.x, c1 * B.x), fma_(m, bb.y, c1 * B.y), m * bb.z};
    return (-q) * axpy(-c3, bxE, w);
}

// state after the classical part of the step, shared by the streaming pass and the event pass
struct LState {
    F3 x, p, s, E, B;
    float gam, w;
    bool qed;
    float chi, lnchi, Wu, Wd, sb, Ws, Wdn;
    F3 khat, eps, beta;
};

// fields at x_old, Boris push, T-BMT precession, move, chi, basis and rates
// ACC: fields from the accurate sine and cosine (the event passes), else the fast ones
template <uint32_t FIX = 0, bool ACC = false>
__device__ __forceinline__ void lepton_classical(const Ctx& C, const float4& a, const float4& b, const float4& cc, LState& st,
                                                 unsigned long long* c,
                                                 const TabP<float>* Tp = nullptr) {
    const TabP<float>& T = Tp ? *Tp : C.T;  // the caller may hand the tables over from its parameters
    const uint32_t fl = flags_of<FIX>(C);
    const float dt = C.S.dt_f;
    const F3 xold{a.x, a.y, a.z};
    st.p = F3{a.w, b.x, b.y};
    st.s = F3{b.z, b.w, cc.x};
    st.w = cc.y;
    constexpr bool PW = plane_waves_only<FIX>();
    field_eval<float, ACC, PW>(C.F, C.S.ph_hi_f, C.S.ph_lo_f, xold, st.E, st.B);
    F3 pb = st.p;  // the time-centred momentum (the push replaces it by its own, cancellation-free form)
    // the field kinds known to have E_z = B_z = 0; any other kind takes the general forms
    const bool transverse = PW || (C.F.kind >= QED_FIELD_LP && C.F.kind <= QED_FIELD_CP_COUNTER);
    if (fl & QED_F_PUSH) st.p = transverse ? boris_t(st.p, st.E, st.B, C.q, dt, pb) : boris32(st.p, st.E, st.B, C.q, dt, pb);
    if (fl & QED_F_TBMT) {
        const bool paper = (fl & QED_F_TBMT_PAPER) != 0;
        // the anomalous moment: alpha/(2 pi), a(chi) at pb, or none (tbmt_a; chi32 takes the plane-wave form)
        float ae = (float)(kAlpha / (2.0 * kPi));
        if (fl & (QED_F_G2 | QED_F_LOOP)) ae = 0.0f;
        else if (fl & QED_F_AMM) ae = amm_lookup(T, chi32<ACC, PW>(C, sqrt_(1.0f + dot(pb, pb)), pb, st.E, st.B, 1.0f, xold).chi);
        st.s = rotate(st.s, transverse ? tbmt_omega_t(pb, st.E, st.B, C.q, paper, ae) : tbmt_omega(pb, st.E, st.B, C.q, paper, ae), dt);
    }
    st.gam = sqrt_(1.0f + dot(st.p, st.p));
    const float rg = rcp_(st.gam);
    st.x = xold;
    if (fl & QED_F_MOVE) {
        st.x = axpy(dt * rg, st.p, xold);
    }
    st.qed = false;
    if (!(fl & QED_F_EMIT)) return;
    const ChiF cf = chi32<ACC, PW>(C, st.gam, st.p, st.E, st.B, 1.0f, xold);
    st.chi = cf.chi;
    const float pn2 = dot(st.p, st.p);
    if (!(pn2 > 0.0f) || !(st.chi > 0.0f) || st.chi < C.S.chi_floor_f) return;
    st.khat = rsqrtf(pn2) * st.p;
    const F3 v = rg * st.p;
    if (!basis32<PW>(C, st.E, st.B, v, st.khat, -C.q, st.eps, st.beta, rg, st.p, 1.0f, cf.f)) return;
    st.qed = true;
    st.lnchi = __logf(st.chi);
    if (c && st.chi > T.chi_max) c[C_CLAMPED]++;
    nlc_rates(T, st.chi, st.lnchi, st.Wu, st.Wd);
    const float pref = (float)(kAlpha / (kSqrt3 * kPi)) * rcp_(C.F.eta0) * rg;
    st.Wu *= pref;
    st.Wd *= pref;
    st.sb = (fl & QED_F_RESOLVED) ? dot(st.s, st.beta) : 0.0f;
    st.Wdn = st.Wd * (1.0f - st.sb) * 0.5f;
    st.Ws = st.Wu * (1.0f + st.sb) * 0.5f + st.Wdn;
}

__device__ __forceinline__ void store32(const PartDev& L, int64_t j, const F3& x, const F3& p, const F3& s, float w, double tau) {
    float lo, hi;
    tau_split(tau, lo, hi);
    L.q0[j] = make_float4(x.x, x.y, x.z, p.x);
    L.q1[j] = make_float4(p.y, p.z, s.x, s.y);
    L.q2[j] = make_float4(s.z, w, lo, hi);
}

// a photon: every plane (a new photon, or one that converted)
__device__ __forceinline__ void store_photon32(const PartDev& G, int64_t j, const F3& x, const F3& k, const F3& P, float w,
                                               double tau) {
    float lo, hi;
    tau_split(tau, lo, hi);
    G.q0[j] = make_float4(x.x, x.y, x.z, P.x);
    G.q1[j] = make_float4(P.y, P.z, lo, hi);
    G.q2[j] = make_float4(k.x, k.y, k.z, w);
}

// a photon step: position, polarization and optical depth (k and w are unchanged)
__device__ __forceinline__ void store_photon32_step(const PartDev& G, int64_t j, const F3& x, const F3& P, double tau) {
    float lo, hi;
    tau_split(tau, lo, hi);
    G.q0[j] = make_float4(x.x, x.y, x.z, P.x);
    G.q1[j] = make_float4(P.y, P.z, lo, hi);
}

// ------------------------------------------------------------------------------------------------
// precision of the event passes
// ------------------------------------------------------------------------------------------------
// An event's outputs are held to FP32 relative precision without the narrow FP64 pipe of this GPU
// wherever that can be done: fields from the accurate sine and cosine (chi keeps its relative precision
// next to a node of the carrier) and the photon's energy fraction from the float-float ICDF lookup
// (ln u' of a soft photon is ~ -40, whose plain FP32 rounding would be ~4e-6 of u').  FP64 is kept for
// the rare parts that need it: every quantity of a pair (pairs are ~2 % of events; their spin
// coefficients 1/(1 - lambda) - xi3/lambda and the like cancel), and the photon's Stokes vector and the
// lepton's spin axis of the events whose FP32 forms cancel (|F| or |g| small against their terms).
struct Tab64 {
    TabP<double> T;     // FP64 rate and ICDF tables
    const double* bes;  // FP64 scaled Bessel table [3][kBesN]
};

__device__ __forceinline__ V3<double> wide(const F3& v) { return V3<double>{v.x, v.y, v.z}; }
__device__ __forceinline__ F3 narrow(const V3<double>& v) { return F3{(float)v.x, (float)v.y, (float)v.z}; }

// An event is taken again in FP64 when |g| or |F| is below this fraction of the sum of the absolute
// values of its terms.  The sum bounds the terms' FP32 rounding from above by a wide margin: measured, the
// direction error of F is ~1e-8 of the sum over |F|, so at this threshold it stays near 1e-6, and only a
// few events in 1e4 (chiefly spin flips against a polarized spin, where F0 = w - |g|) take the FP64 path.
constexpr float kCancel = 0.01f;

// sum over F1, F2, F3 of the absolute values of their terms (App. A.1 Eqs. F1-F3; the Bessel values are
// positive)
__device__ __forceinline__ float nlc_stokes_scale(float lam, float one_m, const float bes[3], const F3& si, const F3& sf,
                                                  const F3& eps, const F3& beta, const F3& k) {
    const float u = div_(lam, one_m);
    const float kappa = rcp_(one_m) + one_m;
    const float kappat = fabsf(rcp_(one_m) - one_m);
    const float K13 = bes[0], K23 = bes[1], IK = bes[2];
    const float sie = fabsf(dot(si, eps)), sib = fabsf(dot(si, beta)), sik = fabsf(dot(si, k));
    const float sfe = fabsf(dot(sf, eps)), sfb = fabsf(dot(sf, beta)), sfk = fabsf(dot(sf, k));
    const F3 fxi = cross(sf, si);
    const float lu2 = 0.5f * lam * u;
    const float A1 = K13 * (u * sie + lam * sfe) + lu2 * IK * (sfe * sib + sfb * sie) + 0.5f * kappat * K23 * fabsf(dot(fxi, k));
    const float A2 = 0.5f * kappat * K13 * fabsf(dot(fxi, eps)) + (lam * IK + kappat * K23) * sik +
                     (u * IK + kappat * K23) * sfk + lu2 * K13 * (sfk * sib + sfb * sik);
    const float A3 = K23 + (u * sib + lam * sfb) * K13 + lu2 * IK * (sfe * sie + sfb * sib) +
                     0.5f * kappa * K23 * fabsf(dot(sf, si)) + lu2 * K23 * sfk * sik;
    return A1 + A2 + A3;
}

// An NLC event taken again in FP64 from the lepton's stored FP32 state (a, b, cc): fields, Boris push,
// T-BMT precession, move, chi and basis, the energy fraction from the FP64 ICDF with the same uniform,
// recoil, the SQA collapse of the spin with r3 and the PQA collapse of the photon's Stokes vector with
// r4 (App. A.1), every flag as the FP64 path reads it.  The FP32 pass calls it for the events whose
// spin axis or photon polarization is ill-conditioned (g or F far below its terms, as after a spin flip
// against a polarized spin: F0 = w - |g|): there the FP32 rounding of the classical step alone, 1e-7 of
// the spin and basis, would move the photon's Stokes vector by up to cond x 1e-7.  The branch (down) is

// Table-free decision by rejection (QED_F_REJECT, Sec. 4.2).  Emission: the candidate lambda = r1^3 is
// accepted with probability 3 r1^2 (dW/dlambda) dt, dW/dlambda = pref w(lambda; s.beta) (App. A.1); pair:
// the candidate positron fraction lambda = r1 with probability (dW/dlambda) dt = pref w0(lambda; xi3) dt
// (App. A.2).  The Bessel values come from the float table (scaled by e^x, unscaled here); beyond x = 80
// the density is below the float range.  A step whose acceptance exceeds 1 is counted (the method needs
// it below 1).
__device__ __forceinline__ bool reject_nlc(const Ctx& C, const uint4& w0, float chi, float gam, float sb,
                                           unsigned long long* c) {
    const float r1 = u52f(w0.x, w0.y), r2 = u52f(w0.z, w0.w);
    const float lc = r1 * r1 * r1, om = 1.0f - lc;
    const float up = div_(2.0f * lc, 3.0f * chi * om);
    if (!(up < 80.0f)) return false;
    float b[3];
    bessel32(C.bes, up, b);
    const float wl = (-b[2] + (rcp_(om) + om) * b[1] + lc * sb * b[0]) * __expf(-up);
    const float acc = 3.0f * r1 * r1 * (float)(kAlpha / (kSqrt3 * kPi)) * rcp_(C.F.eta0 * gam) * wl * C.S.dt_f;
    if (c && acc > 1.0f) c[C_BOUND]++;
    return r2 < acc;
}

__device__ __forceinline__ bool reject_nbw(const Ctx& C, const uint4& w0, float chi, float en, float xi3,
                                           unsigned long long* c) {
    const float r1 = u52f(w0.x, w0.y), r2 = u52f(w0.z, w0.w);
    const float om = 1.0f - r1;
    const float ut = div_(2.0f, 3.0f * chi * r1 * om);
    if (!(ut < 80.0f)) return false;
    float b[3];
    bessel32(C.bes, ut, b);
    const float w0r = (b[2] + (div_(om, r1) + div_(r1, om)) * b[1] - xi3 * b[1]) * __expf(-ut);
    const float acc = (float)(kAlpha / (kSqrt3 * kPi)) * rcp_(C.F.eta0 * en) * w0r * C.S.dt_f;
    if (c && acc > 1.0f) c[C_BOUND]++;
    return r2 < acc;
}

// the FP32 pass's decision.  Outputs: the lepton's x, p, s and the photon's k and P, rounded to float.
static __device__ __noinline__ void lepton_event64(const Ctx& C, const Tab64& X, const FieldP<double>& F64,
                                                  const float4& a, const float4& b, const float4& cc, bool down,
                                                  bool net, float lnu, const uint4& w0, const uint4& w1,
                                                  const uint4& w2, F3& x_out,
                                                  F3& p_out, F3& s_out, F3& k_out, F3& P_out) {
    using V = V3<double>;
    const uint32_t fl = C.S.flags;
    const double dt = C.S.dt, q = (double)C.q;
    V x{a.x, a.y, a.z}, p{a.w, b.x, b.y}, s{b.z, b.w, cc.x};
    V E, B;
    field_eval(F64, C.S.ph_hi, 0.0, x, E, B);
    const V pold = p;
    if (fl & QED_F_PUSH) p = boris(p, E, B, q, dt);
    if (fl & QED_F_TBMT) {
        const V pb = 0.5 * (pold + p);
        s = rotate(s, tbmt_omega(pb, E, B, q, (fl & QED_F_TBMT_PAPER) != 0, tbmt_a(fl, X.T, F64.eta0, pb, E, B)), dt);
    }
    const double gam = sqrt(1.0 + dot(p, p));
    if (fl & QED_F_MOVE) x = x + v3(p.x / gam * dt, p.y / gam * dt, p.z / gam * dt);
    const double chi = chi_of(F64.eta0, gam, p, E, B);
    const double pn = sqrt(dot(p, p));
    const V khat = v3(p.x / pn, p.y / pn, p.z / pn);
    V eps{0, 0, 0}, beta{0, 0, 0};
    make_basis(E, B, v3(p.x / gam, p.y / gam, p.z / gam), khat, -q, eps, beta);
    const double r2 = uniform52(w1.x, w1.y), r3 = uniform52(w1.z, w1.w), r4 = uniform52(w2.x, w2.y);
    double lam, one_m, up;
    if (fl & QED_F_REJECT) {  // the accepted candidate lambda = r1^3
        const double r1 = uniform52(w0.x, w0.y);
        lam = r1 * r1 * r1;
        one_m = 1.0 - lam;
        up = 2.0 * lam / (3.0 * chi * one_m);
    } else if (net) {  // ln u' as the learned sampler drew it from the same uniform r2
        up = exp((double)lnu);
        lam = 3.0 * chi * up / (2.0 + 3.0 * chi * up);
        one_m = 1.0 - lam;
    } else {
        up = exp(icdf_lookup(X.T, false, down ? 1 : 0, log(chi), log(r2) - log(1.0 - r2)));
        lam = 3.0 * chi * up / (2.0 + 3.0 * chi * up);
        one_m = 1.0 - lam;
    }
    const V k = lam * p;
    V pf = p, sf = s, sfu{0, 0, 0}, si{0, 0, 0};
    if (fl & QED_F_RECOIL) pf = one_m * p;
    if (fl & QED_F_RESOLVED) si = s;
    double bb[3];
    bessel64(X.bes, up, bb);
    double xi[3] = {0.0, 0.0, 0.0};
    double wv = 0.0;
    V g{0, 0, 0};
    if (fl & (QED_F_SPIN_EVENT | QED_F_POL_EVENT)) nlc_wg(lam, one_m, bb, si, beta, khat, wv, g);
    if (fl & QED_F_SPIN_EVENT) {
        const double gn = sqrt(dot(g, g));
        if (fl & QED_F_BETA_BASIS) {  // resolved along +-beta (Sec. 8.3 comparison)
            const double gb = dot(g, beta);
            sf = (fl & QED_F_SPIN_COLLAPSE) ? (r3 < (wv - gb) / (2.0 * wv) ? -1.0 : 1.0) * beta : (gb / wv) * beta;
        } else if (fl & QED_F_SPIN_COLLAPSE) {
            const double sg = r3 < (wv - gn) / (2.0 * wv) ? -1.0 : 1.0;
            sf = gn > 0.0 ? v3(sg * g.x / gn, sg * g.y / gn, sg * g.z / gn) : v3(0.0, 0.0, 0.0);
        } else {
            sf = v3(g.x / wv, g.y / wv, g.z / wv);
        }
        sfu = sf;
    }
    if (fl & QED_F_POL_EVENT) {
        double Fv[4];
        nlc_stokes(lam, one_m, bb, si, sfu, wv, g, eps, beta, khat, Fv);
        const double Fn = sqrt(Fv[1] * Fv[1] + Fv[2] * Fv[2] + Fv[3] * Fv[3]);
        if (fl & QED_F_POL_COLLAPSE) {
            const double sg = r4 < (Fv[0] - Fn) / (2.0 * Fv[0]) ? -1.0 : 1.0;
            for (int i = 0; i < 3; ++i) xi[i] = Fn > 0.0 ? sg * Fv[i + 1] / Fn : 0.0;
        } else {
            for (int i = 0; i < 3; ++i) xi[i] = Fv[i + 1] / Fv[0];
        }
    }
    x_out = narrow(x);
    p_out = narrow(pf);
    s_out = narrow(sf);
    k_out = narrow(k);
    P_out = narrow(stokes_to_P(xi, eps, beta, khat));
}

// Events to be taken again in FP64, queued per warp so that the FP64 code runs with all 32 lanes busy
// (one ill-conditioned lane would otherwise make its whole warp run it).  An entry names the lepton, the
// photon's reserved slot (-1: no photon stored), the caller's context key with the branch in bit 30 and
// the learned sampler's ln u' (when the caller uses it).
constexpr int kExactQ = 64;  // entries per warp; drained 32 at a time
struct ExactQ {
    int64_t j[kExactQ];
    int64_t slot[kExactQ];
    int key[kExactQ];
    float lnu[kExactQ];
    int n;
};

// One queued event in FP64 (per lane, not warp-collective): the lepton's stored state is still the one
// the step began with; its event outcome and its photon (in the reserved slot) are written here.
static __device__ __noinline__ void lepton_exact_one(const Ctx& C, const Tab64& X, const FieldP<double>& F64,
                                                    const PartDev& L, const PartDev& G, int64_t j, int64_t slot,
                                                    bool down, bool net = false, float lnu = 0.0f) {
    const uint32_t fl = C.S.flags;
    const float4 a = __ldcg(L.q0 + j), b = __ldcg(L.q1 + j), cc = __ldcg(L.q2 + j);
    const uint64_t id = L.id[j];
    const uint4 w0 = draw(id, C.S.seed, C.S.step, kSlotTauBranch);
    const uint4 w1 = draw(id, C.S.seed, C.S.step, kSlotLambdaSpin);
    const uint4 w2 = draw(id, C.S.seed, C.S.step, kSlotStokes);
    F3 x, pf, sf, k, P;
    lepton_event64(C, X, F64, a, b, cc, down, net, lnu, w0, w1, w2, x, pf, sf, k, P);
    const double tau_new = ((fl & QED_F_TAU) && !(fl & QED_F_REJECT)) ? exp_draw(w0.x, w0.y) : tau_join(cc.z, cc.w);
    store32(L, j, x, pf, sf, cc.y, tau_new);
    if (slot >= 0) {
        const uint4 wc = draw(id, C.S.seed, C.S.step, kSlotChild);
        const uint64_t gid = (uint64_t)wc.x | ((uint64_t)wc.y << 32);
        store_photon32(G, slot, x, k, P, cc.y, birth_tau32(gid, C.S.seed));
        G.id[slot] = gid;
    }
}

// the event pass of one warp (all 32 lanes call it): a lane with j >= 0 takes particle j of buffer L,
// whose step context is C and whose photons go to G through the reservation A (lanes may differ in all
// three; A is NULL when the caller keeps no photons).  q (may be NULL): the warp's queue for the events
// taken again in FP64, with the lane's context key; without it they are taken here.  net: the energy
// fraction is u' = exp(lnu), drawn by the learned sampler from the same uniform (Sec. 5.1), instead of
// the branch's ICDF row.
static __device__ QED_EVENT_PASS void lepton_events(const Ctx& C, const Tab64& X, const FieldP<double>& F64, int64_t j,
                                                 const PartDev& L, const PartDev& G, AppendState* A,
                                                 qed_counters* ctr, unsigned long long* c, ExactQ* q = nullptr,
                                                 int key = 0, bool net = false, float lnu = 0.0f) {
    // The lepton's outcome (energy fraction, recoil, spin) and the photon's polarization for every event,
    // then the photon's slot reservation: an event whose photon does not fit is not applied.
    const uint32_t fl = C.S.flags;
    bool want = false;
    LState st;
    uint64_t id = 0;
    F3 k{0, 0, 0}, pf{0, 0, 0}, sf{0, 0, 0}, P{0, 0, 0};
    float xi[3] = {0.0f, 0.0f, 0.0f};
    double tau_kept = 0.0, tau_new = 0.0;
    bool exact = false;  // the event is taken in FP64 (k, P and the lepton's x, p, s from lepton_event64)
    bool down = false;
    if (j >= 0) {
        const float4 a = __ldcg(L.q0 + j), b = __ldcg(L.q1 + j), cc = __ldcg(L.q2 + j);
        lepton_classical<0, true>(C, a, b, cc, st, nullptr);  // the streaming pass's step, accurate fields
        id = L.id[j];
        pf = st.p;
        sf = st.s;
        // the optical depth as the streaming pass left it (spent), kept if the event is not applied
        const double tau0 = tau_join(cc.z, cc.w);
        const bool rej = (fl & QED_F_REJECT) != 0;
        tau_kept = ((fl & QED_F_TAU) && !rej) ? tau0 - widen_pos(st.Ws * C.S.dt_f) : tau0;
        tau_new = tau_kept;
        const uint4 w0 = draw(id, C.S.seed, C.S.step, kSlotTauBranch);
        if (fl & QED_F_TAU) down = u52f(w0.z, w0.w) * st.Ws < st.Wdn;
        else down = u52f(w0.x, w0.y) < st.Wdn * C.S.dt_f;
        const uint4 w1 = draw(id, C.S.seed, C.S.step, kSlotLambdaSpin);
        const uint4 w2 = draw(id, C.S.seed, C.S.step, kSlotStokes);
        const float r3 = u52f(w1.z, w1.w), r4 = u52f(w2.x, w2.y);
        // the energy fraction to FP32 relative precision (float-float ICDF lookup); FP64 where u' leaves
        // the float range (uniforms within ~1e-10 of 0 or 1)
        float up32;
        double up, lam64, om64;
        if (rej) {  // the accepted candidate lambda = r1^3 (Sec. 4.2)
            const double r1 = uniform52(w0.x, w0.y);
            lam64 = r1 * r1 * r1;
            om64 = 1.0 - lam64;
            up = 2.0 * lam64 / (3.0 * (double)st.chi * om64);
        } else if (net) {
            const double chi = (double)st.chi;
            up = exp((double)lnu);
            const double den = 2.0 + 3.0 * chi * up;
            lam64 = 3.0 * chi * up / den;
            om64 = 2.0 / den;
        } else if (nlc_up_ff(C.T, down ? 1 : 0, logf(st.chi), w1.x, w1.y, up32)) {
            const float den = fmaf(3.0f * st.chi, up32, 2.0f);
            const float iden = rcp_(den);
            lam64 = (double)(3.0f * st.chi * up32 * iden);
            om64 = (double)(2.0f * iden);
            up = (double)up32;
        } else {
            const double r2 = uniform52(w1.x, w1.y), chi = (double)st.chi;
            up = exp(icdf_lookup(X.T, false, down ? 1 : 0, log(chi), log(r2) - log(1.0 - r2)));
            const double den = 2.0 + 3.0 * chi * up;
            lam64 = 3.0 * chi * up / den;
            om64 = 2.0 / den;
        }
        const float lam = (float)lam64, one_m = (float)om64;
        k = lam * st.p;
        if (fl & QED_F_RECOIL) pf = one_m * st.p;
        const F3 si = (fl & QED_F_RESOLVED) ? st.s : F3{0, 0, 0};
        if (fl & (QED_F_SPIN_EVENT | QED_F_POL_EVENT)) {
            float bb[3], wv;
            F3 g;
            bessel32(C.bes, (float)up, bb);
            nlc_wg(lam, one_m, bb, si, st.beta, st.khat, wv, g);
            // the scale of g: the absolute values of its terms (cancellation loses the direction in FP32)
            const float u = div_(lam, one_m);
            const float gs = u * bb[0] + (2.0f * bb[1] + bb[2]) * sqrt_(dot(si, si)) +
                             lam * u * (bb[1] + bb[2]) * fabsf(dot(si, st.khat));
            const float gn = sqrt_(dot(g, g));
            if (!(gn >= kCancel * gs) || !(wv > 0.0f) || !(up >= 1e-30)) {
                exact = true;
            } else {
                F3 sfu{0, 0, 0};
                if (fl & QED_F_SPIN_EVENT) {
                    if (fl & QED_F_BETA_BASIS) {  // resolved along +-beta (Sec. 8.3 comparison)
                        const float gb = dot(g, st.beta);
                        sf = (fl & QED_F_SPIN_COLLAPSE) ? (r3 < div_(wv - gb, 2.0f * wv) ? -1.0f : 1.0f) * st.beta
                                                        : div_(gb, wv) * st.beta;
                    } else if (fl & QED_F_SPIN_COLLAPSE) {
                        const float sg = r3 < div_(wv - gn, 2.0f * wv) ? -1.0f : 1.0f;
                        sf = gn > 0.0f ? div_(sg, gn) * g : F3{0, 0, 0};
                    } else {
                        sf = rcp_(wv) * g;
                    }
                    sfu = sf;
                }
                if (fl & QED_F_POL_EVENT) {
                    float Fv[4];
                    nlc_stokes(lam, one_m, bb, si, sfu, wv, g, st.eps, st.beta, st.khat, Fv);
                    const float Fn = sqrt_(Fv[1] * Fv[1] + Fv[2] * Fv[2] + Fv[3] * Fv[3]);
                    const float Fs = nlc_stokes_scale(lam, one_m, bb, si, sfu, st.eps, st.beta, st.khat);
                    if (!(Fn >= kCancel * Fs)) {
                        exact = true;  // the terms of F cancel (F0 = w - |g| after a spin flip, typically)
                    } else if (fl & QED_F_POL_COLLAPSE) {
                        const float sg = r4 < div_(Fv[0] - Fn, 2.0f * Fv[0]) ? -1.0f : 1.0f;
                        const float iF = div_(sg, Fn);
                        for (int i = 0; i < 3; ++i) xi[i] = Fv[i + 1] * iF;
                    } else {
                        const float iF = rcp_(Fv[0]);
                        for (int i = 0; i < 3; ++i) xi[i] = Fv[i + 1] * iF;
                    }
                }
            }
        }
        if (exact && q == nullptr)
            lepton_event64(C, X, F64, a, b, cc, down, net, lnu, w0, w1, w2, st.x, pf, sf, k, P);
        else if (!exact) P = stokes_to_P(xi, st.eps, st.beta, st.khat);
        if ((fl & QED_F_TAU) && !rej) tau_new = exp_draw(w0.x, w0.y);
        want = sqrt_(dot(k, k)) >= C.S.store_min_f;
        if (!want) c[C_BELOW]++;
    }
    const long long ev = reserve_event(A, want);
    const bool keep = want && A != nullptr && ev < A->budget;
    const bool refused = want && A != nullptr && !keep;
    const bool queued = j >= 0 && exact && q != nullptr && !refused;  // stored by lepton_exact_one later
    if (j >= 0) {
        if (refused) {  // no room for the photon: the event is not applied
            c[C_DROPPED]++;
            record_error(ctr, QED_ERR_CAPACITY, j);
            store32(L, j, st.x, st.p, st.s, st.w, tau_kept);
        } else {
            c[C_EVENTS]++;
            if (want && A == nullptr) c[C_DROPPED]++;  // the caller keeps no photons
            if (!queued) store32(L, j, st.x, pf, sf, st.w, tau_new);
        }
    }
    if (keep) {
        c[C_STORED]++;
        if (!queued) {
            const int64_t slot = A->base[0] + ev;
            const uint4 wc = draw(id, C.S.seed, C.S.step, kSlotChild);
            const uint64_t gid = (uint64_t)wc.x | ((uint64_t)wc.y << 32);
            store_photon32(G, slot, st.x, k, P, st.w, birth_tau32(gid, C.S.seed));
            G.id[slot] = gid;
        }
    }
    if (q != nullptr) {  // warp-uniform
        const unsigned m = __ballot_sync(0xffffffffu, queued);
        if (queued) {
            const int e = q->n + __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
            q->j[e] = j;
            q->slot[e] = keep ? A->base[0] + ev : -1;
            q->key[e] = key | (down ? (1 << 30) : 0);
            q->lnu[e] = lnu;
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) q->n += __popc(m);
        __syncwarp();
    }
}

// the streaming pass of one particle (no event): non-emission update and store; returns true if the
// particle's optical depth ran out (it is then left untouched for the event pass)
template <uint32_t FIX = 0>
__device__ __forceinline__ bool lepton_stream_one(const Ctx& C, const PartDev& L, int64_t j, const float4& a, const float4& b,
                                                  const float4& cc, qed_counters* ctr, unsigned long long* c, const TabP<float>* Tp = nullptr) {
    const uint32_t fl = flags_of<FIX>(C);
    const float dt = C.S.dt_f;
    if (!finite_state(a, b, cc)) {
        c[C_NONFINITE]++;
        record_error(ctr, QED_ERR_NAN, j);
        return false;
    }
    LState st;
    lepton_classical<FIX>(C, a, b, cc, st, c, Tp);
    const double tau = tau_join(cc.z, cc.w);
    double tauf = tau;
    if (st.qed) {
        if (fl & QED_F_REJECT) {
            if (reject_nlc(C, draw(L.id[j], C.S.seed, C.S.step, kSlotTauBranch), st.chi, st.gam, st.sb, c)) return true;
        } else if (fl & QED_F_TAU) {
            tauf = tau - widen_pos(st.Ws * dt);
            if (tau_spent(tauf)) return true;
        } else {
            const uint4 w0 = draw(L.id[j], C.S.seed, C.S.step, kSlotTauBranch);
            if (u52f(w0.x, w0.y) < st.Ws * dt) return true;
        }
    }
    F3 sf = st.s;
    if (st.qed && (fl & QED_F_NONTRANSITION) && (fl & QED_F_RESOLVED)) {
        // Sec. 6: s <- [s (1 - <P> dt) - P_i dt] / [1 - (<P> + P_i . s) dt]
        const float W0 = 0.5f * (st.Wu + st.Wd), Pi = 0.5f * (st.Wu - st.Wd);
        const float D = 1.0f - (W0 + Pi * st.sb) * dt;
        if (D > 0.0f) {
            const float iD = rcp_(D), a1 = (1.0f - W0 * dt) * iD, a2 = Pi * dt * iD;
            sf = axpy(-a2, st.beta, a1 * st.s);
            if (dot(sf, sf) > 1.0f + kRenormSlack) {
                sf = renorm64(sf);
                c[C_RENORM]++;
            }
        }
    }
    if (st.qed && (fl & QED_F_LOOP)) {
        // the loop's Scorer term (App. A.1): a turn about the rest-frame magnetic field
        const TabP<float>& T = Tp ? *Tp : C.T;
        sf = rotate(sf, loop_omega(T, C.F.eta0, st.chi, st.gam, st.p, st.E, st.B, C.q), dt);
    }
    store32(L, j, st.x, st.p, sf, st.w, tauf);
    return false;
}

// ------------------------------------------------------------------------------------------------
// photon step
// ------------------------------------------------------------------------------------------------
struct PState {
    F3 x, k, P, E, B, khat, eps, beta;
    float en, w;
    bool qed;
    float chi, lnchi, xi[3], Wp, Wm, Wmp, Wx;
};

template <uint32_t FIX = 0, bool ACC = false>
__device__ __forceinline__ void photon_classical(const Ctx& C, const float4& a, const float4& b, const float4& cc, PState& st,
                                                 unsigned long long* c,
                                                 const TabP<float>* Tp = nullptr) {
    const TabP<float>& T = Tp ? *Tp : C.T;  // the caller may hand the tables over from its parameters
    const F3 xold{a.x, a.y, a.z};
    st.k = F3{cc.x, cc.y, cc.z};
    st.P = F3{a.w, b.x, b.y};
    st.w = cc.w;
    constexpr bool PW = plane_waves_only<FIX>();
    field_eval<float, ACC, PW>(C.F, C.S.ph_hi_f, C.S.ph_lo_f, xold, st.E, st.B);
    float en2 = dot(st.k, st.k);
    if (en2 < 0x1.0p-100f) {
        // |k|^2 near or below the float range (photons of ~1e-15 mc^2 and softer, a few per 1e8 emissions
        // in the NLC spectrum's lambda^(1/3) tail): the components scaled by 2^100 keep k-hat's precision
        const F3 ks = 0x1.0p+100f * st.k;
        const float e2s = dot(ks, ks);
        st.en = sqrt_(e2s) * 0x1.0p-100f;
        st.khat = e2s > 0.0f ? rsqrtf(e2s) * ks : F3{0, 0, 0};
        en2 = e2s > 0.0f ? fmaxf(en2, 0x1.0p-149f) : 0.0f;  // nonzero exactly when k is
    } else {
        st.en = sqrt_(en2);
        st.khat = rsqrtf(en2) * st.k;
    }
    st.x = xold;
    if (flags_of<FIX>(C) & QED_F_MOVE) st.x = axpy(C.S.dt_f, st.khat, xold);
    st.qed = false;
    if (!(flags_of<FIX>(C) & QED_F_EMIT) || !(en2 > 0.0f)) return;
    const ChiF cf = chi32<ACC, PW>(C, st.en, st.k, st.E, st.B, 0.0f, xold);
    st.chi = cf.chi;
    if (!(st.chi > 0.0f) || st.chi < C.S.chi_floor_f) return;
    st.lnchi = __logf(st.chi);
    if (c && st.chi > T.chi_max) c[C_CLAMPED]++;
    nbw_rates(T, st.chi, st.lnchi, st.Wp, st.Wm);
    // most photons are too soft, or in too weak a field, for a pair rate in the float range: nothing of
    // the basis or the Stokes vector is needed for them (the caller moves them and stops)
    if (st.Wp == 0.0f && st.Wm == 0.0f) return;
    if (!basis32<PW>(C, st.E, st.B, st.khat, st.khat, 1.0f, st.eps, st.beta, rsqrtf(en2), st.k, 0.0f, cf.f)) return;
    st.qed = true;
    P_to_stokes(st.P, st.eps, st.beta, st.khat, st.xi);
    if (!(flags_of<FIX>(C) & QED_F_RESOLVED)) st.xi[0] = st.xi[1] = st.xi[2] = 0.0f;
    const float pref = (float)(kAlpha / (kSqrt3 * kPi)) * rcp_(C.F.eta0 * st.en);
    st.Wp *= pref;
    st.Wm *= pref;
    st.Wmp = st.Wm * (1.0f - st.xi[2]) * 0.5f;
    st.Wx = st.Wp * (1.0f + st.xi[2]) * 0.5f + st.Wmp;
}

// the pair pass of one warp: a lane with j >= 0 takes photon j of G; the pair goes to El and Po through
// the reservation A (NULL: the caller keeps no pairs, and photons do not convert).  Everything after the
// decision is FP64 (pairs are rare; their spin coefficients cancel).
static __device__ QED_EVENT_PASS void photon_events(const Ctx& C, const Tab64& X, int64_t j, const PartDev& G,
                                                 const PartDev& El, const PartDev& Po, AppendState* A,
                                                 qed_counters* ctr, unsigned long long* c) {
    const uint32_t fl = C.S.flags;
    const bool have = A != nullptr;
    bool want = false;
    F3 x{0, 0, 0}, k{0, 0, 0}, P{0, 0, 0}, pe{0, 0, 0}, pp{0, 0, 0}, se{0, 0, 0}, sp{0, 0, 0};
    float w = 0.0f;
    double tauf = 0.0;
    uint64_t ide = 0, idp = 0;
    if (j >= 0) {
        const float4 a = __ldcg(G.q0 + j), b = __ldcg(G.q1 + j), cc = __ldcg(G.q2 + j);
        PState st;
        photon_classical<0, true>(C, a, b, cc, st, nullptr);
        x = st.x;
        k = st.k;
        P = st.P;
        w = st.w;
        tauf = tau_join(b.z, b.w);
        const bool rej = (fl & QED_F_REJECT) != 0;
        if ((fl & QED_F_TAU) && !rej) tauf -= widen_pos(st.Wx * C.S.dt_f);
        const uint64_t id = G.id[j];
        const uint4 w0 = draw(id, C.S.seed, C.S.step, kSlotTauBranch);
        bool minus;
        if (fl & QED_F_TAU) minus = u52f(w0.z, w0.w) * st.Wx < st.Wmp;
        else minus = u52f(w0.x, w0.y) < st.Wmp * C.S.dt_f;
        const uint4 w1 = draw(id, C.S.seed, C.S.step, kSlotLambdaSpin);
        const double r3 = uniform52(w1.z, w1.w);
        // the folded coordinate rf = |2u - 1| = (2 dm + 1) 2^-52 from the integer bits of u, and 1 - rf,
        // both exact in FP64
        const uint64_t m = ((uint64_t)(w1.x >> 12) << 32) | (uint64_t)w1.y;
        const uint64_t half = 1ull << 51;
        const bool low = m < half;  // u < 1/2: the positron takes the smaller fraction
        const uint64_t dm = low ? half - 1ull - m : m - half;
        const double rf = ((double)dm + 0.5) * 0x1.0p-51, rfc = ((double)((half - 1ull) - dm) + 0.5) * 0x1.0p-51;
        const double chi = (double)st.chi;
        double ut, lam, one_m;
        if (rej) {  // the accepted candidate positron fraction lambda = r1 (Sec. 4.2)
            lam = uniform52(w0.x, w0.y);
            one_m = 1.0 - lam;
            ut = 2.0 / (3.0 * chi * lam * one_m);
        } else {
            const double xv = exp(icdf_lookup(X.T, true, minus ? 1 : 0, log(chi), log(rf) - log(rfc)));
            const double umin = (8.0 / 3.0) / chi;
            ut = umin + xv;
            // mu (1 - mu) = q = 2/(3 chi u~'), so 1 - 4q = x/u~' exactly and mu = (1 - sqrt(x/u~'))/2
            // = u~'_min / (2 u~' (1 + sqrt(x/u~'))), free of cancellation near the centre
            const double mu = 0.5 * (umin / ut) / (1.0 + sqrt(xv / ut));
            lam = low ? mu : 1.0 - mu;
            one_m = low ? 1.0 - mu : mu;
        }
        const V3<double> k64 = wide(st.k);
        pp = narrow(lam * k64);
        pe = narrow(one_m * k64);
        if (fl & QED_F_SPIN_EVENT) {
            double bb[3];
            bessel64(X.bes, ut, bb);
            const double xi[3] = {st.xi[0], st.xi[1], st.xi[2]};
            const V3<double> eps = wide(st.eps), beta = wide(st.beta), kh = wide(st.khat);
            double w0v;
            V3<double> je, jp;
            nbw_j(lam, one_m, bb, xi, eps, beta, kh, w0v, je, jp);
            if (fl & QED_F_SPIN_COLLAPSE) {
                const double jen = sqrt(dot(je, je)), jpn = sqrt(dot(jp, jp));
                V3<double> Se = jen > 0.0 ? (1.0 / jen) * je : V3<double>{0, 0, 0};
                V3<double> Sp = jpn > 0.0 ? (1.0 / jpn) * jp : V3<double>{0, 0, 0};
                if (fl & QED_F_BETA_BASIS) Se = Sp = beta;  // the G_ab sum to 4 w0 on any axes
                // four correlated states, order (--, -+, +-, ++), first sign = positron
                double cum = 0.0;
                int chosen = 3;
                for (int s4 = 0; s4 < 3; ++s4) {
                    const double sa = (s4 & 2) ? 1.0 : -1.0, sbb = (s4 & 1) ? 1.0 : -1.0;
                    cum += nbw_G(lam, one_m, bb, xi, sa * Sp, sbb * Se, eps, beta, kh) / (4.0 * w0v);
                    if (r3 < cum) {
                        chosen = s4;
                        break;
                    }
                }
                const double sa = (chosen & 2) ? 1.0 : -1.0, sbb = (chosen & 1) ? 1.0 : -1.0;
                sp = narrow(sa * Sp);
                se = narrow(sbb * Se);
            } else if (fl & QED_F_BETA_BASIS) {
                se = narrow((dot(je, beta) / w0v) * beta);
                sp = narrow((dot(jp, beta) / w0v) * beta);
            } else {
                se = narrow((1.0 / w0v) * je);
                sp = narrow((1.0 / w0v) * jp);
            }
        }
        const uint4 wc = draw(id, C.S.seed, C.S.step, kSlotChild);
        ide = (uint64_t)wc.x | ((uint64_t)wc.y << 32);
        idp = (uint64_t)wc.z | ((uint64_t)wc.w << 32);
        want = true;
    }
    bool ok = false;
    {
        // one reservation for the pair: event ev of the step writes electron base[0] + ev and positron
        // base[1] + ev if ev < budget (both fit), else neither
        const long long ev = reserve_event(A, want);
        ok = want && have && ev < A->budget;
        if (ok) {
            const int64_t s_e = A->base[0] + ev, s_p = A->base[1] + ev;
            store32(El, s_e, x, pe, se, w, birth_tau32(ide, C.S.seed));
            El.id[s_e] = ide;
            store32(Po, s_p, x, pp, sp, w, birth_tau32(idp, C.S.seed));
            Po.id[s_p] = idp;
        }
        const long long s_d = reserve_grouped(have ? G.n_dead : nullptr, ok);
        if (ok && s_d < G.capacity) G.dead[s_d] = j;
    }
    if (want) {
        if (ok) {
            c[C_EVENTS]++;
            c[C_STORED] += 2;
            store_photon32(G, j, x, F3{0, 0, 0}, P, 0.0f, tauf);  // converted: inert until compaction
        } else {
            c[C_DROPPED]++;
            if (have) record_error(ctr, QED_ERR_CAPACITY, j);
            store_photon32_step(G, j, x, P, tauf);  // survives and retries next step
        }
    }
}

template <uint32_t FIX = 0>
__device__ __forceinline__ bool photon_stream_one(const Ctx& C, const PartDev& G, int64_t j, const float4& a, const float4& b,
                                                  const float4& cc, qed_counters* ctr, unsigned long long* c, const TabP<float>* Tp = nullptr) {
    const uint32_t fl = flags_of<FIX>(C);
    const float dt = C.S.dt_f;
    if (!finite_photon(a, b, cc)) {
        c[C_NONFINITE]++;
        record_error(ctr, QED_ERR_NAN, j);
        return false;
    }
    PState st;
    photon_classical<FIX>(C, a, b, cc, st, c, Tp);
    if (!st.qed) {
        // no pair rate here (outside the pulse, or W_+ and W_- below the float range): the optical depth
        // stays, the non-pair update is the identity and P, k, w do not change, so only the position
        // plane is written (16 of the photon's 48 bytes)
        G.q0[j] = make_float4(st.x.x, st.x.y, st.x.z, a.w);
        return false;
    }
    const double tau = tau_join(b.z, b.w);
    double tauf = tau;
    if (st.qed && (fl & QED_F_REJECT)) {
        if (reject_nbw(C, draw(G.id[j], C.S.seed, C.S.step, kSlotTauBranch), st.chi, st.en, st.xi[2], c)) return true;
    } else if (st.qed && st.Wx > 0.0f) {
        if (fl & QED_F_TAU) {
            tauf = tau - widen_pos(st.Wx * dt);
            if (tau_spent(tauf)) return true;
        } else {
            const uint4 w0 = draw(G.id[j], C.S.seed, C.S.step, kSlotTauBranch);
            if (u52f(w0.x, w0.y) < st.Wx * dt) return true;
        }
    }
    F3 Pf = st.P;
    if (st.qed && (fl & QED_F_NONTRANSITION) && (fl & QED_F_RESOLVED)) {
        // Sec. 6 with Q = e3: xi <- [xi (1 - <P> dt) - P_i dt e3] / [1 - (<P> + P_i xi3) dt]
        const float W0 = 0.5f * (st.Wp + st.Wm), Pi = 0.5f * (st.Wp - st.Wm);
        const float D = 1.0f - (W0 + Pi * st.xi[2]) * dt;
        if (D > 0.0f) {
            const float iD = rcp_(D), a1 = (1.0f - W0 * dt) * iD;
            float xn[3] = {st.xi[0] * a1, st.xi[1] * a1, st.xi[2] * a1 - Pi * dt * iD};
            if (xn[0] * xn[0] + xn[1] * xn[1] + xn[2] * xn[2] > 1.0f + kRenormSlack) {
                const F3 r = renorm64(F3{xn[0], xn[1], xn[2]});
                xn[0] = r.x;
                xn[1] = r.y;
                xn[2] = r.z;
                c[C_RENORM]++;
            }
            Pf = stokes_to_P(xn, st.eps, st.beta, st.khat);
        }
    }
    store_photon32_step(G, j, st.x, Pf, tauf);
    c[C_RATE_STEPS]++;
    return false;
}

}  // namespace qed
