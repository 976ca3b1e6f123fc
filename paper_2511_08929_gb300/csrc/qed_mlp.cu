// qed_mlp.cu -- the learned sampler: a 3-64-64-64-4 SiLU network standing in for the three-dimensional
// inverse CDF in (chi, r, s_beta) that Sec. 5.1 rejects for its memory.
//
// Target (the map the network learns, computed from the FP64 tables): the exact r-quantile ln u' of the
// NLC spectrum for a continuous spin projection s (w is linear in s: the mixture CDF is the rate-weighted
// blend of the two branch CDFs, each the inverse of its interpolated ICDF row) and the photon Stokes
// vector there (App. A.1, s_i = s beta_hat, final spin summed: xi1 = xi2 = 0, xi3 = F3/F0).  The network
// predicts the correction to the rate-weighted blend of the two branch quantiles (and of xi3 there),
// scaled by 100.
//
// Kernels: target generation (FP64), a BF16 GEMM on the tensor cores (tcgen05.mma, FP32 accumulator in
// TMEM; split-K for the weight gradients), FP32 elementwise / first-layer / reduction / AdamW kernels for
// training, and a fused inference kernel (layers 2-4 as tcgen05.mma on 128-sample tiles, bias and SiLU
// between them applied on the way from TMEM back to shared memory), followed by the CDF check and the
// table fallback.
#include <cstring>

#include <cuda_bf16.h>

#include "qed_device.cuh"
#include "qed_internal.h"

namespace qed {

// ---- parameter layout (FP32, one array): W1[64][3] b1[64] W2[64][64] b2 W3[64][64] b3 W4[4][64] b4[4]
constexpr int kH = 64;
constexpr int kOffW1 = 0, kOffB1 = 192, kOffW2 = 256, kOffB2 = 4352, kOffW3 = 4416, kOffB3 = 8512, kOffW4 = 8576,
              kOffB4 = 8832, kParams = 8836;
static_assert(kParams == QED_MLP_PARAMS, "parameter count");

constexpr double kLnChiLo = -6.907755278982137, kLnChiHi = 4.605170185988092;  // ln 1e-3, ln 1e2
constexpr double kYClamp = 20.0;
constexpr double kOutScale = 100.0;
constexpr uint64_t kMlpStep = 0xFFFFFFFFFFFFFFFEull;  // reserved Philox step of the training inputs

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// ---- the map from (chi, r, s) to the target, FP64 tables -------------------------------------------
template <class R>
struct MixPointT {
    R lnchi, y, s, a;  // a = (1 + s) I_up / ((1 + s) I_up + (1 - s) I_down)
    R qu, qd;          // the two branch quantiles at the logit y
};
using MixPoint = MixPointT<double>;

__device__ inline MixPoint mix_point(const TabP<double>& T, double chi, double r, double s) {
    MixPoint m;
    m.lnchi = log(chi);
    m.y = log(r) - log1p(-r);
    m.s = s;
    double Iu, Id;
    nlc_rates(T, chi, m.lnchi, Iu, Id);
    m.a = (1.0 + s) * Iu / ((1.0 + s) * Iu + (1.0 - s) * Id);
    m.qu = icdf_lookup(T, false, 0, m.lnchi, m.y);
    m.qd = icdf_lookup(T, false, 1, m.lnchi, m.y);
    return m;
}

// the same point on the float tables; the logit from r and 1 - r, each rounded to float once, so that
// neither end of (0, 1) loses its precision
__device__ inline MixPointT<float> mix_point32(const TabP<float>& T, double chi, double r, double s) {
    MixPointT<float> m;
    const float c = (float)chi, sf = (float)s;
    m.lnchi = logf(c);
    m.y = logf((float)r) - logf((float)(1.0 - r));
    m.s = sf;
    float Iu, Id;
    nlc_rates(T, c, m.lnchi, Iu, Id);
    m.a = (1.0f + sf) * Iu / ((1.0f + sf) * Iu + (1.0f - sf) * Id);
    m.qu = icdf_lookup(T, false, 0, m.lnchi, m.y);
    m.qd = icdf_lookup(T, false, 1, m.lnchi, m.y);
    return m;
}

// Root of a monotone increasing g on the bracket [a, c] (g(a) < 0 < g(c)) by regula falsi with the
// Illinois weight (the end that stays put has its value halved, so neither end stalls), started at the
// guess x0; a step outside the bracket falls back to its midpoint.  Stops when the bracket is below
// dx or |g| below dg, after at most ITERS evaluations.
template <int ITERS, class R, class G>
__device__ inline R illinois(G g, R a, R ga, R c, R gc, R x0, R dx, R dg) {
    R x = x0 < a ? a : (x0 > c ? c : x0);
    if (!(x > a && x < c)) x = R(0.5) * (a + c);
    int side = 0;
    for (int it = 0; it < ITERS; ++it) {
        const R f = g(x);
        if ((f < R(0) ? -f : f) <= dg) return x;
        if (f < R(0)) {
            a = x;
            ga = f;
            if (side == -1) gc *= R(0.5);
            side = -1;
        } else {
            c = x;
            gc = f;
            if (side == 1) ga *= R(0.5);
            side = 1;
        }
        if (c - a <= dx) break;
        x = (a * gc - c * ga) / (gc - ga);
        if (!(x > a && x < c)) x = R(0.5) * (a + c);
    }
    return R(0.5) * (a + c);
}

// CDF of one spin branch at ln u' = L: the logit y at which the interpolated ICDF row equals L, mapped
// to r.  The search starts at the mixture point's logit yg, whose quantile qg is known: steps of
// (L - qg)/3 (the slope of ln u' in the logit below the grid; it is smaller above), doubled until the
// sign of ICDF(y) - L changes, bracket the root, and the solver finishes inside the bracket.  A step
// that reaches an end of the grid without the change means L lies beyond the tabulated range: above it
// the CDF is 1, below it the linear asymptote is inverted directly.  In FP64 (R = double) the logit to
// 1e-10, so the CDF to 3e-11; on the float tables the logit to 1e-6 and the CDF to ~3e-7 (the float
// entries' own rounding, ~6e-8 of ln u', adds no more than that).
template <int ITERS, class R>
__device__ inline R branch_cdf(const TabP<R>& T, int b, R lnchi, R L, R yg, R qg) {
    constexpr bool F64 = sizeof(R) == 8;
    const R yhi = T.y_lo + R(T.n_r - 1) / T.inv_dy;
    auto g = [&](R yy) { return icdf_lookup(T, false, b, lnchi, yy) - L; };
    const R g0 = qg - L;
    if (g0 == R(0)) return R(1) / (R(1) + exp_(-yg));
    const bool up = g0 < R(0);  // the root lies above yg
    R x = yg, gx = g0;
    R step = (L - qg) / R(3);
    step = step < R(0) ? -step : step;
    if (step < R(F64 ? 1e-9 : 1e-5)) step = R(F64 ? 1e-9 : 1e-5);
    R a = x, ga = gx, c = x, gc = gx;
    bool found = false;
    for (int k = 0; k < 26 && !found; ++k) {
        R xn = up ? x + step : x - step;
        const bool edge = up ? xn >= yhi : xn <= T.y_lo;
        if (edge) xn = up ? yhi : T.y_lo;
        const R gn = g(xn);
        if (up ? gn >= R(0) : gn <= R(0)) {
            a = up ? x : xn;
            ga = up ? gx : gn;
            c = up ? xn : x;
            gc = up ? gn : gx;
            found = true;
        } else if (edge) {
            if (up) return R(1);                                   // L above the row's last entry
            return R(1) / (R(1) + exp_(-(T.y_lo + (-gn) / R(3))));  // below: y_lo + (L - bottom)/3
        } else {
            x = xn;
            gx = gn;
            step *= R(2);
        }
    }
    if (!found) return R(1) / (R(1) + exp_(-x));  // not reached: 26 doublings span the grid
    const R aL = L < R(0) ? -L : L;
    const R x0 = a - ga * (c - a) / (gc - ga);
    const R y = illinois<ITERS>(g, a, ga, c, gc, x0, R(F64 ? 1e-10 : 1e-6), R(F64 ? 1e-13 : 1e-7) * (aL > R(1) ? aL : R(1)));
    return R(1) / (R(1) + exp_(-y));
}

// the mixture's CDF at L: each branch solved from the mixture point's own logit, near which its root
// lies (at most ITERS evaluations each)
template <int ITERS, class R>
__device__ inline R mix_cdf(const TabP<R>& T, const MixPointT<R>& m, R L) {
    return m.a * branch_cdf<ITERS>(T, 0, m.lnchi, L, m.y, m.qu) +
           (R(1) - m.a) * branch_cdf<ITERS>(T, 1, m.lnchi, L, m.y, m.qd);
}

// the blend of the two branch quantiles (the baseline the network corrects)
template <class R>
__device__ inline R mix_baseline(const TabP<R>& T, const MixPointT<R>& m) {
    return m.a * m.qu + (R(1) - m.a) * m.qd;
}

// the exact mixture quantile: the mixture CDF lies between the branch CDFs, so its quantile lies between
// the branch quantiles; the same solver there, from the blend of the two, until the mixture CDF is
// within 2e-11 of r (the inner solves' own accuracy) or the bracket below 1e-12 in ln u'
template <int OUTER, int INNER>
__device__ inline double mix_quantile(const TabP<double>& T, const MixPoint& m, double r) {
    const double qu = m.qu, qd = m.qd;
    const double lo = fmin(qu, qd) - 1e-9, hi = fmax(qu, qd) + 1e-9;
    auto g = [&](double L) { return mix_cdf<INNER>(T, m, L) - r; };
    const double glo = g(lo), ghi = g(hi);
    if (!(glo < 0.0)) return lo;
    if (!(ghi > 0.0)) return hi;
    return illinois<OUTER>(g, lo, glo, hi, ghi, m.a * qu + (1.0 - m.a) * qd, 1e-12, 2e-11);
}

// xi3 = F3 / F0 at u' for s_i = s beta_hat, s_f = 0 (App. A.1)
__device__ inline double xi3_at(const double* __restrict__ bes_tab, double chi, double L, double s) {
    // a network output outside any physical range (or not finite) never reaches the Bessel evaluation
    if (!(L > -200.0 && L < 50.0)) return nan("");
    const double up = exp(L);
    const double lam = 3.0 * chi * up / (2.0 + 3.0 * chi * up), one_m = 1.0 - lam;
    double b[3];
    bessel64(bes_tab, up, b);
    const double u = lam / one_m, kappa = 1.0 / one_m + one_m;
    return (b[1] + u * s * b[0]) / (-b[2] + kappa * b[1] + lam * s * b[0]);
}

// the same from the float Bessel table
__device__ inline float xi3_at32(const float* __restrict__ bes32, float chi, float L, float s) {
    if (!(L > -85.0f && L < 50.0f)) return __int_as_float(0x7FC00000);  // u' outside the float range
    const float up = expf(L);
    const float den = fmaf(3.0f * chi, up, 2.0f), lam = 3.0f * chi * up / den, one_m = 2.0f / den;
    float b[3];
    bessel32(bes32, up, b);
    const float u = lam / one_m, kappa = 1.0f / one_m + one_m;
    return (b[1] + u * s * b[0]) / (-b[2] + kappa * b[1] + lam * s * b[0]);
}

__device__ inline void mlp_features(double chi, double r, double s, float x[3]) {
    const double y = fmin(kYClamp, fmax(-kYClamp, log(r) - log1p(-r)));
    x[0] = (float)((log(chi) - 0.5 * (kLnChiLo + kLnChiHi)) / (0.5 * (kLnChiHi - kLnChiLo)));
    x[1] = (float)(y / 10.0);
    x[2] = (float)s;
}

__global__ void mlp_targets_kernel(TabP<double> T, const double* __restrict__ bes_tab, int64_t n, uint64_t seed,
                                   int64_t first, float* __restrict__ X, float* __restrict__ Y, double* __restrict__ raw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t id = (uint64_t)(first + i);
        const uint4 w0 = draw(id, seed, kMlpStep, 0), w1 = draw(id, seed, kMlpStep, 1);
        const double lnchi = kLnChiLo + uniform52(w0.x, w0.y) * (kLnChiHi - kLnChiLo);
        const double chi = exp(lnchi), r = uniform52(w0.z, w0.w), s = 2.0 * uniform52(w1.x, w1.y) - 1.0;
        const MixPoint m = mix_point(T, chi, r, s);
        const double Lb = mix_baseline(T, m), L = mix_quantile<44, 32>(T, m, r);
        float x[3];
        mlp_features(chi, r, s, x);
        X[3 * i] = x[0];
        X[3 * i + 1] = x[1];
        X[3 * i + 2] = x[2];
        Y[4 * i] = (float)(kOutScale * (L - Lb));
        Y[4 * i + 1] = 0.0f;
        Y[4 * i + 2] = 0.0f;
        Y[4 * i + 3] = (float)(kOutScale * (xi3_at(bes_tab, chi, L, s) - xi3_at(bes_tab, chi, Lb, s)));
        if (raw) {
            raw[3 * i] = chi;
            raw[3 * i + 1] = r;
            raw[3 * i + 2] = s;
        }
    }
}

// ---- BF16 helpers -------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (lower 16 bits), .y = hi
    return *reinterpret_cast<const uint32_t*>(&v);
}

// ---- training kernels (FP32) ------------------------------------------------------------------------
// layer 1: Z1 = X W1^T + b1, H1 = silu(Z1)
__global__ void mlp_layer1_kernel(const float* __restrict__ P, const float* __restrict__ X, int64_t n, float* Z,
                                  float* H) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kH; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / kH;
        const int j = (int)(e % kH);
        const float* w = P + kOffW1 + 3 * j;
        const float z = fmaf(w[0], X[3 * b], fmaf(w[1], X[3 * b + 1], fmaf(w[2], X[3 * b + 2], P[kOffB1 + j])));
        Z[e] = z;
        H[e] = silu_f(z);
    }
}

// Z += bias (in place), H = silu(Z)
__global__ void mlp_bias_silu_kernel(const float* __restrict__ bias, int64_t n, float* Z, float* H) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kH; e += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[e] + bias[e % kH];
        Z[e] = z;
        H[e] = silu_f(z);
    }
}

// O += b4; dO = 2 (O - T) / n; loss += sum (O - T)^2 / n
__global__ void mlp_out_loss_kernel(const float* __restrict__ P, const float* __restrict__ Tg, int64_t n, float* O,
                                    float* dO, float* loss) {
    float acc = 0.0f;
    const float inv = 1.0f / (float)n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * 4; e += (int64_t)gridDim.x * blockDim.x) {
        const float o = O[e] + P[kOffB4 + (e & 3)];
        O[e] = o;
        const float d = o - Tg[e];
        dO[e] = 2.0f * d * inv;
        acc = fmaf(d * inv, d, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc);
}

// dZ = dH * silu'(Z) (in place on dH)
__global__ void mlp_silu_back_kernel(const float* __restrict__ Z, int64_t n, float* dH) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kH; e += (int64_t)gridDim.x * blockDim.x)
        dH[e] *= dsilu_f(Z[e]);
}

// column sums of D[n][w] into out[w] (one block per column; deterministic order)
__global__ void mlp_colsum_kernel(const float* __restrict__ D, int64_t n, int w, float* out) {
    __shared__ float red[32];
    const int col = blockIdx.x;
    float acc = 0.0f;
    for (int64_t b = threadIdx.x; b < n; b += blockDim.x) acc += D[b * w + col];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) out[col] = acc;
    }
}

// dW1[j][i] = sum_b dZ1[b][j] X[b][i] (one block per entry, FP32)
__global__ void mlp_dw1_kernel(const float* __restrict__ dZ, const float* __restrict__ X, int64_t n, float* g) {
    __shared__ float red[32];
    const int j = blockIdx.x / 3, i = blockIdx.x % 3;
    float acc = 0.0f;
    for (int64_t b = threadIdx.x; b < n; b += blockDim.x) acc = fmaf(dZ[b * kH + j], X[3 * b + i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) g[kOffW1 + 3 * j + i] = acc;
    }
}

__device__ __forceinline__ bool is_weight(int k) {
    return k < kOffB1 || (k >= kOffW2 && k < kOffB2) || (k >= kOffW3 && k < kOffB3) || (k >= kOffW4 && k < kOffB4);
}

// AdamW (decoupled weight decay on weights only); t = step count after this update
__global__ void mlp_adamw_kernel(float* P, float* Mm, float* Vv, const float* __restrict__ G, float lr, float wd,
                                 float b1t, float b2t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kParams) return;
    const float g = G[k];
    const float m = 0.9f * Mm[k] + 0.1f * g;
    const float v = 0.999f * Vv[k] + 0.001f * g * g;
    Mm[k] = m;
    Vv[k] = v;
    const float mh = m / (1.0f - b1t), vh = v / (1.0f - b2t);
    float upd = mh / (sqrtf(vh) + 1e-8f);
    if (is_weight(k)) upd += wd * P[k];
    P[k] -= lr * upd;
}

// ---- fused inference on the 5th-generation tensor cores ---------------------------------------------
// A block of 128 threads takes 128 samples at a time, one per thread and one per TMEM lane.  Layer 1
// (K = 3) runs in FP32 on the CUDA cores; each thread writes its 64 SiLU outputs as BF16 into the A
// tile in shared memory; one thread issues the 128 x 64 x 64 layer as four tcgen05.mma (K = 16 each)
// with the FP32 accumulator in TMEM and commits them to an mbarrier; every thread then reads its row
// of the accumulator (tcgen05.ld), adds the bias, applies SiLU and writes the next layer's A row.  The
// output layer is padded to 16 rows (the smallest MMA width at M = 128).  Operands are K-major without
// swizzle: core matrices of 8 rows x 16 bytes, 128 bytes apart along K, 8-row groups 1024 bytes apart.
constexpr int kIW = 4;         // warps per block
constexpr int kTR = kIW * 32;  // samples per tile (the MMA's M)
constexpr int kTN4 = 16;       // output layer rows after padding
constexpr uint32_t kTmemCols = 64;
constexpr int kTcWaitLimit = 1 << 24;  // bounded mbarrier polling (~0.1 s) before giving up

struct TcShared {
    alignas(1024) unsigned char a[kTR * kH * 2];  // activations (A operand), 16 KB
    alignas(1024) unsigned char w2[kH * kH * 2];  // W2, W3 as B operands (N = 64 rows of K = 64)
    alignas(1024) unsigned char w3[kH * kH * 2];
    alignas(1024) unsigned char w4[kTN4 * kH * 2];  // W4 padded to 16 rows
    float w1[kOffW2];                               // W1, b1 (FP32)
    float b2[kH], b3[kH], b4[4];
    int64_t queue[2 * kTR];  // sampler: indices of samples waiting for the table path
    int queued;
    uint64_t bar;            // MMA completion
    uint32_t tmem;           // TMEM base address of the accumulator
};

// byte offset of element (row r, column k) in a K-major tile with K = 64
__device__ __forceinline__ uint32_t kmaj(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t sm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (8-row group) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTR >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// the 16 accumulator columns c0.. of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// D = A W^T for the A tile and the B operand w (n rows): thread 0 issues, every thread waits.  Returns
// false (in every thread) if the wait gave up.
__device__ bool tc_layer(TcShared& S, const unsigned char* w, int n, uint32_t& phase) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the A rows written above, to the MMA
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t id = tc_idesc(n);
#pragma unroll
        for (int ks = 0; ks < kH / 16; ++ks) {
            const uint64_t da = tc_desc(sm_u32(S.a) + 256 * ks), db = tc_desc(sm_u32(w) + 256 * ks);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(S.tmem),
                "l"(da), "l"(db), "r"(id), "r"((uint32_t)ks)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_u32(&S.bar))
                     : "memory");
    }
    bool done = false;
    for (int i = 0; i < kTcWaitLimit && !done; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(sm_u32(&S.bar)), "r"(phase)
            : "memory");
        done = ok != 0;
    }
    phase ^= 1u;
    tc_fence_after();
    return __syncthreads_and(done) != 0;
}

// this thread's 64 activations, bias + SiLU, into its A row as BF16
__device__ __forceinline__ void tc_store_row(TcShared& S, const float v[kH]) {
    const int r = threadIdx.x;
#pragma unroll
    for (int c = 0; c < kH / 8; ++c) {
        uint4 q;
        q.x = pack_bf16(v[8 * c], v[8 * c + 1]);
        q.y = pack_bf16(v[8 * c + 2], v[8 * c + 3]);
        q.z = pack_bf16(v[8 * c + 4], v[8 * c + 5]);
        q.w = pack_bf16(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4*>(S.a + kmaj(r, 8 * c)) = q;
    }
}

// layers 1-4 for this thread's features x; o = raw outputs.  False if the tensor cores did not answer.
__device__ bool tc_infer(TcShared& S, const float x[3], uint32_t& phase, float o[4]) {
    float v[kH];
#pragma unroll
    for (int k = 0; k < kH; ++k) {
        const float* w = S.w1 + 3 * k;
        v[k] = silu_f(fmaf(w[0], x[0], fmaf(w[1], x[1], fmaf(w[2], x[2], S.w1[kOffB1 + k]))));
    }
    tc_store_row(S, v);
    const uint32_t lane_addr = S.tmem + ((uint32_t)(threadIdx.x & ~31) << 16);
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
        if (!tc_layer(S, layer == 0 ? S.w2 : S.w3, kH, phase)) return false;
        const float* bias = layer == 0 ? S.b2 : S.b3;
#pragma unroll
        for (int c0 = 0; c0 < kH; c0 += 16) tc_ld16(lane_addr + (uint32_t)c0, v + c0);
#pragma unroll
        for (int k = 0; k < kH; ++k) v[k] = silu_f(v[k] + bias[k]);
        tc_store_row(S, v);
    }
    if (!tc_layer(S, S.w4, kTN4, phase)) return false;
    float u[16];
    tc_ld16(lane_addr, u);
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = u[j] + S.b4[j];
    return true;
}

// weights into shared memory, the mbarrier, and the TMEM accumulator (warp 0)
__device__ void tc_setup(TcShared& S, const float* __restrict__ P) {
    const int tid = threadIdx.x;
    for (int i = tid; i < kOffW2; i += blockDim.x) S.w1[i] = P[i];
    for (int i = tid; i < kH; i += blockDim.x) {
        S.b2[i] = P[kOffB2 + i];
        S.b3[i] = P[kOffB3 + i];
    }
    if (tid < 4) S.b4[tid] = P[kOffB4 + tid];
    for (int i = tid; i < kH * kH; i += blockDim.x) {
        const int r = i / kH, k = i % kH;
        *reinterpret_cast<__nv_bfloat16*>(S.w2 + kmaj(r, k)) = __float2bfloat16_rn(P[kOffW2 + i]);
        *reinterpret_cast<__nv_bfloat16*>(S.w3 + kmaj(r, k)) = __float2bfloat16_rn(P[kOffW3 + i]);
    }
    for (int i = tid; i < kTN4 * kH; i += blockDim.x) {
        const int r = i / kH, k = i % kH;
        *reinterpret_cast<__nv_bfloat16*>(S.w4 + kmaj(r, k)) = __float2bfloat16_rn(r < 4 ? P[kOffW4 + i] : 0.0f);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_u32(&S.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(&S.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ void tc_teardown(uint32_t tmem) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---- BF16 GEMM on the tensor cores for training (FP32 in global memory, rounded to BF16 when staged;
// FP32 accumulation in TMEM) ----------------------------------------------------------------------------
// C(m, n) (+)= sum_k A(m, k) B(k, n); A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn]; C row-major
// with leading dimension ldc.  A block of 128 threads computes a 128 x 64 tile of C, staging 64-wide K
// slices of A and B (any strides) as K-major BF16 operands and accumulating with tcgen05.mma.
// grid = (ceil(N/64), ceil(M/128), ksplit); with ksplit > 1 the partial sums are added atomically (C
// zeroed by the caller).  If the tensor cores do not answer within the wait limit the tile is NaN.
struct GemmShared {
    alignas(1024) unsigned char a[kTR * kH * 2];  // A slice: 128 rows x 64 K
    alignas(1024) unsigned char b[kH * kH * 2];   // B slice: 64 columns of C x 64 K
    uint64_t bar;
    uint32_t tmem;
};

__global__ void __launch_bounds__(kTR) gemm_bf16_kernel(int M, int N, int K, const float* __restrict__ A, int64_t sam,
                                                         int64_t sak, const float* __restrict__ B, int64_t sbk,
                                                         int64_t sbn, float* __restrict__ C, int64_t ldc, int ksplit) {
    __shared__ GemmShared S;
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_u32(&S.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(&S.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int m0 = blockIdx.y * kTR, n0 = blockIdx.x * kH;
    const int kchunk = ((K + ksplit - 1) / ksplit + kH - 1) / kH * kH;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const uint32_t id = tc_idesc(kH);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = kb; k0 < ke && ok; k0 += kH) {
        for (int e = tid; e < kTR * kH; e += kTR) {
            const int mm = e / kH, kk = e % kH, m = m0 + mm, k = k0 + kk;
            *reinterpret_cast<__nv_bfloat16*>(S.a + kmaj(mm, kk)) =
                __float2bfloat16_rn(m < M && k < ke ? A[m * sam + k * sak] : 0.0f);
        }
        for (int e = tid; e < kH * kH; e += kTR) {
            const int nn = e / kH, kk = e % kH, n = n0 + nn, k = k0 + kk;
            *reinterpret_cast<__nv_bfloat16*>(S.b + kmaj(nn, kk)) =
                __float2bfloat16_rn(n < N && k < ke ? B[k * sbk + n * sbn] : 0.0f);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks) {
                const uint64_t da = tc_desc(sm_u32(S.a) + 256 * ks), db = tc_desc(sm_u32(S.b) + 256 * ks);
                const uint32_t acc = (k0 > kb || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(S.tmem),
                    "l"(da), "l"(db), "r"(id), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             sm_u32(&S.bar))
                         : "memory");
        }
        bool done = false;
        for (int i = 0; i < kTcWaitLimit && !done; ++i) {
            uint32_t r;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(r)
                : "r"(sm_u32(&S.bar)), "r"(phase)
                : "memory");
            done = r != 0;
        }
        phase ^= 1u;
        tc_fence_after();
        ok = __syncthreads_and(done) != 0;  // also: the slices may be restaged
    }
    if (kb < ke) {
        const int m = m0 + tid;
        const uint32_t lane_addr = S.tmem + ((uint32_t)(tid & ~31) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tc_ld16(lane_addr + (uint32_t)c0, v);
            if (m < M)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < N) {
                        const float x = ok ? v[j] : __int_as_float(0x7FC00000);
                        if (ksplit > 1) atomicAdd(&C[m * ldc + n], x);
                        else C[m * ldc + n] = x;
                    }
                }
        }
    }
    tc_teardown(S.tmem);
}

// raw network outputs for feature rows X[n][3] (NaN where the tensor cores did not answer)
__global__ void __launch_bounds__(kTR) mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                          int64_t n, float* __restrict__ O) {
    __shared__ TcShared S;
    tc_setup(S, P);
    uint32_t phase = 0;
    bool broken = false;  // a wait gave up: the remaining tiles skip the network (the same in every thread)
    for (int64_t base = (int64_t)blockIdx.x * kTR; base < n; base += (int64_t)gridDim.x * kTR) {
        const int64_t i = base + threadIdx.x;
        float x[3] = {0.0f, 0.0f, 0.0f}, o[4];
        if (i < n)
            for (int q = 0; q < 3; ++q) x[q] = X[3 * i + q];
        broken = broken || !tc_infer(S, x, phase, o);
        if (broken)
            for (int j = 0; j < 4; ++j) o[j] = __int_as_float(0x7FC00000);
        if (i < n)
            for (int j = 0; j < 4; ++j) O[4 * i + j] = o[j];
    }
    tc_teardown(S.tmem);
}

// flags bit of the sampling kernel for callers that use ln u' only (the batched step's event pass):
// no Stokes outputs, so neither their check nor xi3 on the table path
constexpr int kLnUpOnly = 4;

// the table path for sample i (the exact mixture quantile, and xi3 there unless ln_up_only)
__device__ void table_path(const TabP<double>& T, const double* __restrict__ bes_tab, const double* __restrict__ chi_in,
                           const double* __restrict__ r_in, const double* __restrict__ s_in, int64_t i,
                           float* __restrict__ out4, bool ln_up_only) {
    const double chi = chi_in[i], r = r_in[i], s = s_in[i];
    const MixPoint m = mix_point(T, chi, r, s);
    const double L = mix_quantile<44, 32>(T, m, r);
    out4[4 * i] = (float)L;
    out4[4 * i + 1] = 0.0f;
    out4[4 * i + 2] = 0.0f;
    out4[4 * i + 3] = ln_up_only ? 0.0f : (float)xi3_at(bes_tab, chi, L, s);
}

// The check of a network sample, first on the float tables: the FP32 CDF and xi3 errors are within ~1e-6
// of the FP64 ones, so a sample whose FP32 errors are below tol - kMargin32 passes and one with an error
// above tol + kMargin32 fails without FP64 work; only samples in the band between are checked again on
// the FP64 tables (the FP64 pipe of this GPU runs at 1/64 of the FP32 rate).
constexpr float kMargin32 = 1e-5f;

// the sampler: network, CDF check; samples that fail it (or all, flags bit 0) wait in a block-wide queue
// and take the table path 128 at a time, one per thread, so that the block never waits on a few slow
// threads (the tiles of the network keep the block in step)
__global__ void __launch_bounds__(kTR) mlp_sample_kernel(const float* __restrict__ P, TabP<double> T,
                                                         TabP<float> T32, const float* __restrict__ bes32,
                                                         const double* __restrict__ bes_tab,
                                                         const double* __restrict__ chi_in, const double* __restrict__ r_in,
                                                         const double* __restrict__ s_in, int64_t n, double tol,
                                                         int flags, float* __restrict__ out4, uint8_t* __restrict__ fell,
                                                         float* __restrict__ err_out, unsigned long long* n_fallback,
                                                         const unsigned long long* __restrict__ n_dev = nullptr) {
    __shared__ TcShared S;
    if (n_dev) {  // a count the previous kernel of the stream left on the device
        const int64_t nd = (int64_t)*n_dev;
        if (nd < n) n = nd;
    }
    if (threadIdx.x == 0) S.queued = 0;
    tc_setup(S, P);
    unsigned long long nf = 0;  // thread 0: fallbacks of this block
    uint32_t phase = 0;
    bool broken = false;  // a wait gave up: the remaining tiles take the table path (the same in every thread)
    const bool table_only = (flags & 1) != 0;
    const bool ln_up_only = (flags & kLnUpOnly) != 0;
    for (int64_t base = (int64_t)blockIdx.x * kTR; base < n; base += (int64_t)gridDim.x * kTR) {
        const int64_t i = base + threadIdx.x;
        float x[3] = {0.0f, 0.0f, 0.0f}, o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (i < n) mlp_features(chi_in[i], r_in[i], s_in[i], x);
        bool net = false;  // the network ran for this tile
        if (!table_only && !broken) {
            net = tc_infer(S, x, phase, o);
            broken = !net;
        }
        if (i < n) {
            bool fb = !net;
            if (!fb) {
                const double chi = chi_in[i], r = r_in[i], s = s_in[i];
                // the sample on the float tables: baseline, correction, CDF error (and xi3's)
                const MixPointT<float> m32 = mix_point32(T32, chi, r, s);
                const float Lb = mix_baseline(T32, m32);
                const float L = Lb + o[0] / (float)kOutScale;
                float xi1 = 0.0f, xi2 = 0.0f, xi3 = 0.0f, dxi3 = 0.0f;
                if (!ln_up_only) {
                    xi1 = o[1] / (float)kOutScale;
                    xi2 = o[2] / (float)kOutScale;
                    xi3 = xi3_at32(bes32, (float)chi, Lb, (float)s) + o[3] / (float)kOutScale;
                    dxi3 = fabsf(xi3 - xi3_at32(bes32, (float)chi, L, (float)s));
                }
                const float ftol = (float)tol;
                float err_q = fabsf(mix_cdf<30>(T32, m32, L) - (float)r);  // the CDF check
                const bool stokes_ok = fabsf(xi1) <= ftol && fabsf(xi2) <= ftol;
                const bool pass32 = err_q <= ftol - kMargin32 && dxi3 <= ftol - kMargin32 && stokes_ok;
                const bool fail32 = !(err_q <= ftol + kMargin32) || !(dxi3 <= ftol + kMargin32) || !stokes_ok;
                fb = !pass32;
                if (!pass32 && !fail32) {  // the band around tol: the FP64 check decides
                    const MixPoint m = mix_point(T, chi, r, s);
                    const double e64 = fabs(mix_cdf<30>(T, m, (double)L) - r);
                    double d64 = 0.0;
                    if (!ln_up_only)
                        d64 = fabs(xi3_at(bes_tab, chi, mix_baseline(T, m), s) + (double)o[3] / kOutScale -
                                   xi3_at(bes_tab, chi, (double)L, s));
                    err_q = (float)e64;
                    fb = !(e64 <= tol) || !(d64 <= tol);
                }
                if (err_out) err_out[i] = err_q;
                if (!fb) {
                    out4[4 * i] = L;
                    out4[4 * i + 1] = xi1;
                    out4[4 * i + 2] = xi2;
                    out4[4 * i + 3] = xi3;
                }
            } else if (err_out) {
                err_out[i] = -1.0f;
            }
            if (fell) fell[i] = fb ? 1 : 0;
            if (fb) S.queue[atomicAdd(&S.queued, 1)] = i;  // at most 2 kTR - 1 entries
        }
        __syncthreads();
        const int qn = S.queued;  // the same in every thread
        if (qn >= kTR) {
            table_path(T, bes_tab, chi_in, r_in, s_in, S.queue[qn - kTR + threadIdx.x], out4, ln_up_only);
            __syncthreads();
            if (threadIdx.x == 0) {
                S.queued = qn - kTR;
                nf += kTR;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    const int qn = S.queued;
    if ((int)threadIdx.x < qn) table_path(T, bes_tab, chi_in, r_in, s_in, S.queue[threadIdx.x], out4, ln_up_only);
    if (threadIdx.x == 0 && n_fallback && nf + (unsigned long long)qn) atomicAdd(n_fallback, nf + (unsigned long long)qn);
    tc_teardown(S.tmem);
}

// The method the network would replace, as the step's event pass runs it (Sec. 5.1): the spin branch
// taken with probability W_down (1 - s)/(2 W_s), the uniform rescaled within the chosen branch (the pair
// gives the mixture w(lambda; s) exactly, reading C4), one row of that branch's ICDF in float-float
// (nlc_up_ff, the FP64 row where u' leaves the float range), and xi3 at the sampled u' from the float
// Bessel table.  out4 = (ln u', 0, 0, xi3).
__global__ void branch_table_kernel(TabP<float> T, TabP<double> T64, const float* __restrict__ bes32,
                                    const double* __restrict__ chi_in, const double* __restrict__ r_in,
                                    const double* __restrict__ s_in, int64_t n, float* __restrict__ out4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float chi = (float)chi_in[i], s = (float)s_in[i];
        const double r = r_in[i];
        const float lnchi = logf(chi);
        float Iu, Id;
        nlc_rates(T, chi, lnchi, Iu, Id);
        const double wd = (double)Id * (1.0 - s) * 0.5, wu = (double)Iu * (1.0 + s) * 0.5;
        const double pd = wd / (wu + wd);
        const bool down = r < pd;
        double rr = down ? r / pd : (r - pd) / (1.0 - pd);
        rr = fmin(fmax(rr, 0x1.0p-53), 1.0 - 0x1.0p-53);
        uint64_t m = (uint64_t)(rr * 0x1.0p52);
        if (m > (1ull << 52) - 1ull) m = (1ull << 52) - 1ull;
        const uint32_t whi = (uint32_t)(m >> 32) << 12, wlo = (uint32_t)m;
        float up;
        if (!nlc_up_ff(T, down ? 1 : 0, lnchi, whi, wlo, up)) {
            const double u = uniform52(whi, wlo);
            up = (float)exp(icdf_lookup(T64, false, down ? 1 : 0, (double)lnchi, log(u) - log(1.0 - u)));
        }
        const float den = fmaf(3.0f * chi, up, 2.0f), lam = 3.0f * chi * up / den, one_m = 2.0f / den;
        float b[3];
        bessel32(bes32, up, b);
        const float u = lam / one_m, kappa = 1.0f / one_m + one_m;
        out4[4 * i] = logf(up);
        out4[4 * i + 1] = 0.0f;
        out4[4 * i + 2] = 0.0f;
        out4[4 * i + 3] = (b[1] + u * s * b[0]) / (-b[2] + kappa * b[1] + lam * s * b[0]);
    }
}

}  // namespace qed

// ---- host side -------------------------------------------------------------------------------------
using namespace qed;

constexpr uint32_t kMlpMagic = 0x514D4C50u;  // "QMLP"

struct qed_mlp_s {
    uint32_t magic;
    int64_t max_batch;
    float *P, *M, *V, *G;  // parameters, Adam moments, gradients
    float *X, *T, *Z1, *H1, *Z2, *H2, *Z3, *H3, *O, *dO, *dA, *dB, *loss;
    int64_t steps;         // AdamW steps taken
};

static bool valid_mlp(const qed_mlp_s* m) { return m && m->magic == kMlpMagic; }

static int grid_for(int64_t work, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 16));
}

static void gemm(int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbk,
                 int64_t sbn, float* C, int64_t ldc, int ksplit, cudaStream_t st) {
    const dim3 grid((N + kH - 1) / kH, (M + kTR - 1) / kTR, ksplit);
    gemm_bf16_kernel<<<grid, kTR, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, ksplit);
}

extern "C" void qed_mlp_destroy(qed_mlp_t m) {
    if (!valid_mlp(m)) return;
    for (float* p : {m->P, m->M, m->V, m->G, m->X, m->T, m->Z1, m->H1, m->Z2, m->H2, m->Z3, m->H3, m->O, m->dO, m->dA,
                     m->dB, m->loss})
        cudaFree(p);
    m->magic = 0;
    delete m;
}

extern "C" qed_status qed_mlp_create(int64_t max_batch, const float* init_params, qed_mlp_t* out) {
    if (!out || max_batch < 1 || max_batch > (1ll << 26) || !init_params) return QED_ERR_ARG;
    *out = nullptr;
    qed_mlp_s* m = new qed_mlp_s();
    m->magic = kMlpMagic;
    m->max_batch = max_batch;
    const size_t np = sizeof(float) * kParams, nb = (size_t)max_batch;
    bool ok = cudaMalloc(&m->P, np) == cudaSuccess && cudaMalloc(&m->M, np) == cudaSuccess &&
              cudaMalloc(&m->V, np) == cudaSuccess && cudaMalloc(&m->G, np) == cudaSuccess &&
              cudaMalloc(&m->X, 3 * nb * 4) == cudaSuccess && cudaMalloc(&m->T, 4 * nb * 4) == cudaSuccess;
    for (float** p : {&m->Z1, &m->H1, &m->Z2, &m->H2, &m->Z3, &m->H3, &m->dA, &m->dB})
        ok = ok && cudaMalloc(p, kH * nb * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&m->O, 4 * nb * 4) == cudaSuccess && cudaMalloc(&m->dO, 4 * nb * 4) == cudaSuccess &&
         cudaMalloc(&m->loss, 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        qed_mlp_destroy(m);
        return QED_ERR_NOMEM;
    }
    if (cudaMemcpy(m->P, init_params, np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->M, 0, np) != cudaSuccess || cudaMemset(m->V, 0, np) != cudaSuccess) {
        qed_mlp_destroy(m);
        return QED_ERR_CUDA;
    }
    *out = m;
    return QED_OK;
}

extern "C" qed_status qed_mlp_get_params(qed_mlp_t m, float* host_out) {
    if (!valid_mlp(m)) return QED_ERR_STATE;
    if (!host_out) return QED_ERR_ARG;
    return cudaMemcpy(host_out, m->P, sizeof(float) * kParams, cudaMemcpyDeviceToHost) == cudaSuccess ? QED_OK
                                                                                                    : QED_ERR_CUDA;
}

extern "C" qed_status qed_mlp_set_params(qed_mlp_t m, const float* host_in) {
    if (!valid_mlp(m)) return QED_ERR_STATE;
    if (!host_in) return QED_ERR_ARG;
    if (cudaMemcpy(m->P, host_in, sizeof(float) * kParams, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->M, 0, sizeof(float) * kParams) != cudaSuccess ||
        cudaMemset(m->V, 0, sizeof(float) * kParams) != cudaSuccess)
        return QED_ERR_CUDA;
    m->steps = 0;
    return QED_OK;
}

extern "C" qed_status qed_mlp_targets(qed_tables_t t, int64_t n, uint64_t seed, int64_t first_index, float* x_dev,
                                      float* y_dev, double* raw_dev, void* stream) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    if (n < 0 || first_index < 0 || (n > 0 && (!x_dev || !y_dev))) return QED_ERR_ARG;
    if (n == 0) return QED_OK;
    mlp_targets_kernel<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(tab_params<double>(t), t->bes64, n, seed,
                                                                         first_index, x_dev, y_dev, raw_dev);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

// forward and backward of one batch (features x, targets y); gradients into grad (kParams floats)
static void mlp_grad_launch(qed_mlp_s* m, const float* x, const float* y, int64_t n, float* grad, float* loss,
                            cudaStream_t st) {
    const float* P = m->P;
    const int eg = grid_for(n * kH, 256);
    const int ks = (int)std::min<int64_t>(64, std::max<int64_t>(1, n / 512));
    mlp_layer1_kernel<<<eg, 256, 0, st>>>(P, x, n, m->Z1, m->H1);
    gemm((int)n, kH, kH, m->H1, kH, 1, P + kOffW2, 1, kH, m->Z2, kH, 1, st);
    mlp_bias_silu_kernel<<<eg, 256, 0, st>>>(P + kOffB2, n, m->Z2, m->H2);
    gemm((int)n, kH, kH, m->H2, kH, 1, P + kOffW3, 1, kH, m->Z3, kH, 1, st);
    mlp_bias_silu_kernel<<<eg, 256, 0, st>>>(P + kOffB3, n, m->Z3, m->H3);
    gemm((int)n, 4, kH, m->H3, kH, 1, P + kOffW4, 1, kH, m->O, 4, 1, st);
    if (loss) cudaMemsetAsync(loss, 0, sizeof(float), st);
    mlp_out_loss_kernel<<<grid_for(n * 4, 256), 256, 0, st>>>(P, y, n, m->O, m->dO, loss);
    cudaMemsetAsync(grad, 0, sizeof(float) * kParams, st);
    // layer 4
    gemm(4, kH, (int)n, m->dO, 1, 4, m->H3, kH, 1, grad + kOffW4, kH, ks, st);
    mlp_colsum_kernel<<<4, 256, 0, st>>>(m->dO, n, 4, grad + kOffB4);
    gemm((int)n, kH, 4, m->dO, 4, 1, P + kOffW4, kH, 1, m->dA, kH, 1, st);
    mlp_silu_back_kernel<<<eg, 256, 0, st>>>(m->Z3, n, m->dA);
    // layer 3
    gemm(kH, kH, (int)n, m->dA, 1, kH, m->H2, kH, 1, grad + kOffW3, kH, ks, st);
    mlp_colsum_kernel<<<kH, 256, 0, st>>>(m->dA, n, kH, grad + kOffB3);
    gemm((int)n, kH, kH, m->dA, kH, 1, P + kOffW3, kH, 1, m->dB, kH, 1, st);
    mlp_silu_back_kernel<<<eg, 256, 0, st>>>(m->Z2, n, m->dB);
    // layer 2
    gemm(kH, kH, (int)n, m->dB, 1, kH, m->H1, kH, 1, grad + kOffW2, kH, ks, st);
    mlp_colsum_kernel<<<kH, 256, 0, st>>>(m->dB, n, kH, grad + kOffB2);
    gemm((int)n, kH, kH, m->dB, kH, 1, P + kOffW2, kH, 1, m->dA, kH, 1, st);
    mlp_silu_back_kernel<<<eg, 256, 0, st>>>(m->Z1, n, m->dA);
    // layer 1 (FP32)
    mlp_dw1_kernel<<<3 * kH, 256, 0, st>>>(m->dA, x, n, grad);
    mlp_colsum_kernel<<<kH, 256, 0, st>>>(m->dA, n, kH, grad + kOffB1);
}

extern "C" qed_status qed_mlp_grad(qed_mlp_t m, const float* x_dev, const float* y_dev, int64_t n, float* grad_dev,
                                   float* loss_dev, void* stream) {
    if (!valid_mlp(m)) return QED_ERR_STATE;
    if (n < 1 || n > m->max_batch || !x_dev || !y_dev || !grad_dev) return QED_ERR_ARG;
    mlp_grad_launch(m, x_dev, y_dev, n, grad_dev, loss_dev, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_mlp_adamw(qed_mlp_t m, const float* grad_dev, float lr, float weight_decay, void* stream) {
    if (!valid_mlp(m)) return QED_ERR_STATE;
    if (!grad_dev || !(lr >= 0.0f) || !(weight_decay >= 0.0f)) return QED_ERR_ARG;
    m->steps += 1;
    const float b1t = (float)std::pow(0.9, (double)m->steps), b2t = (float)std::pow(0.999, (double)m->steps);
    mlp_adamw_kernel<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m->P, m->M, m->V, grad_dev, lr,
                                                                               weight_decay, b1t, b2t);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_mlp_train(qed_mlp_t m, qed_tables_t t, int64_t steps, int64_t batch, uint64_t seed,
                                    int64_t first_index, float lr, float lr_final, float weight_decay,
                                    float* loss_per_step_dev, void* stream) {
    if (!valid_mlp(m)) return QED_ERR_STATE;
    if (!valid_tables(t)) return QED_ERR_STATE;
    if (steps < 0 || batch < 1 || batch > m->max_batch || first_index < 0 || !(lr >= 0.0f) || !(lr_final >= 0.0f))
        return QED_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t k = 0; k < steps; ++k) {
        // cosine decay from lr to lr_final
        const double c = steps > 1 ? 0.5 * (1.0 + std::cos(3.141592653589793 * (double)k / (double)(steps - 1))) : 1.0;
        const float lrk = (float)(lr_final + (lr - lr_final) * c);
        qed_status s = qed_mlp_targets(t, batch, seed, first_index + k * batch, m->X, m->T, nullptr, stream);
        if (s != QED_OK) return s;
        mlp_grad_launch(m, m->X, m->T, batch, m->G, loss_per_step_dev ? loss_per_step_dev + k : nullptr, st);
        s = qed_mlp_adamw(m, m->G, lrk, weight_decay, stream);
        if (s != QED_OK) return s;
    }
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

// persistent grid for the tensor-core kernels: one resident wave of 128-thread blocks, at most 4 per SM
// (each holds 64 TMEM columns of the SM's 512, and its 38 KB of shared memory)
static int tc_blocks(int64_t n, const void* kern) {
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTR, 0);
    const int64_t resident = (int64_t)sms * std::max(1, std::min(per_sm, 4));
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kTR - 1) / kTR, resident));
}

extern "C" qed_status qed_mlp_forward(qed_mlp_t m, const float* x_dev, int64_t n, float* out_dev, void* stream) {
    if (!valid_mlp(m)) return QED_ERR_STATE;
    if (n < 0 || (n > 0 && (!x_dev || !out_dev))) return QED_ERR_ARG;
    if (n == 0) return QED_OK;
    mlp_forward_kernel<<<tc_blocks(n, (const void*)mlp_forward_kernel), kTR, 0, (cudaStream_t)stream>>>(m->P, x_dev, n,
                                                                                                   out_dev);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_mlp_sample(qed_mlp_t m, qed_tables_t t, const double* chi, const double* r, const double* s,
                                     int64_t n, double tol, int32_t flags, float* out4, uint8_t* fell_back,
                                     float* err_out, unsigned long long* n_fallback, void* stream) {
    if (!valid_mlp(m)) return QED_ERR_STATE;
    if (!valid_tables(t)) return QED_ERR_STATE;
    if (n < 0 || (n > 0 && (!chi || !r || !s || !out4)) || !(tol >= 0.0) ||
        (flags & ~(QED_MLP_ALWAYS_TABLE | QED_MLP_BRANCH_TABLE)))
        return QED_ERR_ARG;
    if (n == 0) return QED_OK;
    if (flags & QED_MLP_BRANCH_TABLE) {
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 152 * 16);
        branch_table_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(tab_params<float>(t), tab_params<double>(t),
                                                                          t->bes32, chi, r, s, n, out4);
        return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
    }
    // persistent grid (one resident wave): each warp streams many 32-sample rows, so its fallback queue
    // drains full
    const int blocks = tc_blocks(n, (const void*)mlp_sample_kernel);
    mlp_sample_kernel<<<blocks, kTR, 0, (cudaStream_t)stream>>>(m->P, tab_params<double>(t), tab_params<float>(t),
                                                                t->bes32, t->bes64, chi, r, s, n, tol, flags, out4,
                                                                fell_back, err_out, n_fallback);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

// ---- the sampler inside the batched step (qed_batch.cu) ------------------------------------------------

bool mlp_valid(qed_mlp_t m) { return valid_mlp(m); }

int mlp_listed_grid(int64_t n_max) { return tc_blocks(n_max, (const void*)mlp_sample_kernel); }

qed_status mlp_sample_listed(qed_mlp_t m, const qed_tables_s* t, const double* chi, const double* r, const double* s,
                             int64_t n_max, const unsigned long long* n_dev, double tol, float* out4,
                             unsigned long long* n_fallback, int grid, cudaStream_t st) {
    mlp_sample_kernel<<<grid, kTR, 0, st>>>(m->P, tab_params<double>(t), tab_params<float>(t), t->bes32, t->bes64,
                                            chi, r, s, n_max, tol, kLnUpOnly, out4, nullptr, nullptr, n_fallback,
                                            n_dev);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}
