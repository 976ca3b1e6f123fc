// qed_tables.cu -- FP64 construction of the rate and inverse-CDF tables of Sec. 5.1 (W_up, W_down,
// IntF^-1_up/down) and Sec. 5.2 (W_+, W_-, IntG^-1_+/-), from the Bessel forms of App. A.
//
// Every stored number is an exact (to FP64 rounding) value of a defined integral or of the root of a
// monotone equation; the quadrature is only the means:
//   NLC, variable t with u' = t^3 (removes the lambda^{-2/3} infrared behaviour noted in Sec. 4.2):
//       density in t  = w_s(lambda) d lambda/dt,  lambda = 3 chi u'/(2 + 3 chi u'),
//       d lambda/du' = 6 chi / (2 + 3 chi u')^2,  w_s = -IntK13 + kappa K23 + s lambda K13 at u'.
//   NBW, spectrum folded about lambda = 1/2 (it is symmetric), variable t with u~' = 8/(3 chi) + t^2:
//       density in t of one half = w0_s(u~') * 4 / (3 chi u~'^{3/2}), w0_s = IntK13 + rho K23 - s K23,
//       rho = 3 chi u~'/2 - 2; stored scaled by e^{8/(3 chi)}.
// Each row integrates panels of width 1/16 in t with 12-point Gauss-Legendre, sums them into the
// CDF at the panel edges, and inverts the CDF at each r_m by Newton's method inside the bracketing
// panel (partial integrals again by 12-point Gauss-Legendre).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "qed_bessel.cuh"
#include "qed_internal.h"

namespace qed {

constexpr int kGL = 12;
constexpr double kPanel = 1.0 / 16.0;
__constant__ double c_gl_x[kGL];
__constant__ double c_gl_w[kGL];

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on the Legendre recurrence.
static void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

__global__ void bessel_table_kernel(double* tab64, float* tab32) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kBesN) return;
    const double x = exp(log(kBesLo) + kBesH * j);
    double o[3];
    bessel_trapezoid(x, o);
    for (int f = 0; f < 3; ++f) {
        tab64[f * kBesN + j] = o[f];
        tab32[f * kBesN + j] = (float)o[f];
    }
}

__device__ __forceinline__ double row_density(const double* __restrict__ bes, bool nbw, double chi, double sigma, double t) {
    double b[3];
    if (!nbw) {
        const double up = t * t * t;
        const double den = 2.0 + 3.0 * chi * up;
        const double lam = 3.0 * chi * up / den, one_m = 2.0 / den;
        bessel64(bes, up, b);
        const double kappa = 1.0 / one_m + one_m;
        const double w = exp(-up) * (-b[2] + kappa * b[1] + sigma * lam * b[0]);
        return w * 6.0 * chi / (den * den) * 3.0 * t * t;
    }
    const double ut = 8.0 / (3.0 * chi) + t * t;
    bessel64(bes, ut, b);
    const double rho = 1.5 * chi * ut - 2.0;
    const double w0 = b[2] + rho * b[1] - sigma * b[1];
    return w0 * exp(-t * t) * 4.0 / (3.0 * chi * ut * sqrt(ut));
}

__device__ __forceinline__ double gl_integral(const double* bes, bool nbw, double chi, double sigma, double a, double b) {
    const double m = 0.5 * (a + b), r = 0.5 * (b - a);
    double s = 0.0;
#pragma unroll 4
    for (int i = 0; i < kGL; ++i) s += c_gl_w[i] * row_density(bes, nbw, chi, sigma, m + r * c_gl_x[i]);
    return s * r;
}

constexpr int kMaxPanels = 160;  // sqrt(80) * 16 = 143.1 -> 144 panels for NBW, 69 for NLC

// one block per (kind, sign, chi row)
__global__ void __launch_bounds__(256) table_rows_kernel(const double* __restrict__ bes, qed_table_desc d, double* rates,
                                                         double* icdf) {
    __shared__ double cum[kMaxPanels + 1];
    const int n_chi = d.n_chi;
    const int job = blockIdx.x;
    const bool nbw = job >= 2 * n_chi;
    const int s = (job / n_chi) % 2;
    const int i = job % n_chi;
    const double sigma = s == 0 ? 1.0 : -1.0;
    const double dl = (log(d.chi_max) - log(d.chi_min)) / (n_chi - 1);
    const double chi = exp(log(d.chi_min) + i * dl);
    const double tend = nbw ? sqrt(80.0) : cbrt(80.0);
    const int np = (int)ceil(tend / kPanel);
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const double a = p * kPanel, b = fmin(tend, (p + 1) * kPanel);
        cum[p + 1] = gl_integral(bes, nbw, chi, sigma, a, b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cum[0] = 0.0;
        for (int p = 0; p < np; ++p) cum[p + 1] += cum[p];
        const double total = cum[np];
        rates[(nbw ? 2 * n_chi : 0) + s * n_chi + i] = nbw ? log(2.0 * total) : log(total);
    }
    __syncthreads();
    const double total = cum[np];
    const double dy = (d.y_hi - d.y_lo) / (d.n_r - 1);
    double* out = icdf + ((size_t)((nbw ? 2 : 0) + s) * n_chi + i) * d.n_r;
    for (int m = threadIdx.x; m < d.n_r; m += blockDim.x) {
        const double y = d.y_lo + m * dy;
        const double r = 1.0 / (1.0 + exp(-y));
        const double target = r * total;
        // panel with cum[p] <= target < cum[p+1]
        int lo = 0, hi = np - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cum[mid] <= target) lo = mid; else hi = mid - 1;
        }
        const int p = lo;
        const double a = p * kPanel, b = fmin(tend, (p + 1) * kPanel);
        double tl = a, th = b;
        double t = a + (b - a) * (target - cum[p]) / (cum[p + 1] - cum[p]);
        for (int it = 0; it < 100; ++it) {
            const double F = cum[p] + gl_integral(bes, nbw, chi, sigma, a, t) - target;
            if (F > 0.0) th = t; else tl = t;
            const double dF = row_density(bes, nbw, chi, sigma, t);
            double tn = t - F / dF;
            if (!(tn > tl && tn < th)) tn = 0.5 * (tl + th);
            const bool done = fabs(tn - t) <= 1e-15 * fmax(t, 1e-300) || th - tl <= 1e-15 * th;
            t = tn;
            if (done) break;
        }
        out[m] = nbw ? 2.0 * log(t) : 3.0 * log(t);
    }
}

__global__ void to_float_kernel(const double* __restrict__ a, float* b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// a as the unevaluated float sum hi + lo (hi = a rounded to float, lo = the rest rounded to float)
__global__ void split_float_kernel(const double* __restrict__ a, float* hi, float* lo, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float h = (float)a[i];
        hi[i] = h;
        lo[i] = (float)(a[i] - (double)h);
    }
}

// ------------------------------------------------------------------------------------------------
// field-dependent anomalous moment (the one-loop Scorer term of App. A.1; g(chi) of Sec. 8.6.2)
// ------------------------------------------------------------------------------------------------
// Scorer function for z >= 0 from its defining integral pi Gi(z) = Im int_0^inf exp(i(z t + t^3/3)) dt,
// taken along the ray t = e^{i pi/6} s (the integrand is analytic and bounded between the two rays):
//   pi Gi(z) = int_0^inf exp(-s^3/3 - z s/2) sin(sqrt(3) z s/2 + pi/6) ds,
// a decaying integrand with at most ~13 oscillations before the exponential falls below e^-46:
// 40 panels of 12-point Gauss-Legendre on [0, min(5.2, 92/z)].
__device__ double scorer_gi(double z) {
    const double S = fmin(5.2, 92.0 / fmax(z, 1e-300));
    constexpr int np = 40;
    const double h = S / np, w = 0.86602540378443864676 * z, r = 0.5 * h;
    double acc = 0.0;
    for (int p = 0; p < np; ++p) {
        const double m = (p + 0.5) * h;
        double ps = 0.0;
        for (int i = 0; i < kGL; ++i) {
            const double t = m + r * c_gl_x[i];
            ps += c_gl_w[i] * exp(-t * t * t / 3.0 - 0.5 * z * t) * sin(w * t + kPi / 6.0);
        }
        acc += ps * r;
    }
    return acc / kPi;
}

// One block per chi node: a(chi) = (alpha/chi) int_0^inf du u/(1+u)^3 Gi(z)/sqrt(z), z = (u/chi)^{2/3}
// (= (alpha/chi) int_0^1 dlambda lambda Gi(z)/sqrt(z) with u = lambda/(1-lambda)), integrated in x = ln u
// on [min(ln chi, 0) - 21, max(ln chi, 0) + 21] (the ends add below 1e-17 of the result) with panels of
// width 1/4, one per thread, summed in a fixed tree order.  Stores ln a.
__global__ void __launch_bounds__(256) amm_table_kernel(qed_table_desc d, double* amm64, float* amm32) {
    __shared__ double part[256];
    const int i = blockIdx.x;
    const double dl = (log(d.chi_max) - log(d.chi_min)) / (d.n_chi - 1);
    const double lnchi = log(d.chi_min) + i * dl, chi = exp(lnchi);
    const double x0 = fmin(lnchi, 0.0) - 21.0, x1 = fmax(lnchi, 0.0) + 21.0;
    const int np = (int)ceil((x1 - x0) * 4.0);
    const double h = (x1 - x0) / np, r = 0.5 * h;
    double acc = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const double m = x0 + (p + 0.5) * h;
        for (int k = 0; k < kGL; ++k) {
            const double x = m + r * c_gl_x[k];
            const double u = exp(x);
            const double sz = exp((x - lnchi) / 3.0);  // sqrt(z) = (u/chi)^{1/3}
            const double q = 1.0 / (1.0 + u);
            acc += c_gl_w[k] * r * u * u * q * q * q * scorer_gi(sz * sz) / sz;
        }
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double la = log(kAlpha / chi * part[0]);
        amm64[i] = la;
        amm32[i] = (float)la;
    }
}

}  // namespace qed

using namespace qed;

static void free_tables(qed_tables_s* t) {
    if (!t) return;
    cudaFree(t->rate64);
    cudaFree(t->icdf64);
    cudaFree(t->rate32);
    cudaFree(t->icdf32);
    cudaFree(t->icdf32lo);
    cudaFree(t->bes64);
    cudaFree(t->bes32);
    cudaFree(t->amm64);
    cudaFree(t->amm32);
    t->magic = 0;
    delete t;
}

extern "C" qed_status qed_tables_build(const qed_table_desc* desc, qed_tables_t* out, void* stream) {
    if (!desc || !out) return QED_ERR_ARG;
    const qed_table_desc d = *desc;
    if (d.n_chi < 2 || d.n_r < 4 || d.n_chi > (1 << 16) || d.n_r > (1 << 16) || !(d.chi_min > 0.0) ||
        !(d.chi_max > d.chi_min) || !(d.y_hi > d.y_lo) || !std::isfinite(d.chi_max) || !std::isfinite(d.y_lo) ||
        !std::isfinite(d.y_hi))
        return QED_ERR_ARG;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    qed_tables_s* t = new qed_tables_s();
    std::memset(t, 0, sizeof(*t));
    t->desc = d;
    cudaGetDevice(&t->device);
    const size_t nr = 4 * (size_t)d.n_chi, ni = 4 * (size_t)d.n_chi * d.n_r;
    bool ok = cudaMalloc(&t->rate64, nr * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&t->icdf64, ni * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&t->rate32, nr * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&t->icdf32, ni * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&t->icdf32lo, ni * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&t->bes64, 3 * kBesN * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&t->bes32, 3 * kBesN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&t->amm64, d.n_chi * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&t->amm32, d.n_chi * sizeof(float)) == cudaSuccess;
    if (!ok) {
        free_tables(t);
        return QED_ERR_NOMEM;
    }
    double glx[kGL], glw[kGL];
    gauss_legendre(kGL, glx, glw);
    if (cudaMemcpyToSymbolAsync(c_gl_x, glx, sizeof(glx), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_gl_w, glw, sizeof(glw), 0, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        free_tables(t);
        return QED_ERR_CUDA;
    }
    bessel_table_kernel<<<(kBesN + 127) / 128, 128, 0, st>>>(t->bes64, t->bes32);
    table_rows_kernel<<<4 * d.n_chi, 256, 0, st>>>(t->bes64, d, t->rate64, t->icdf64);
    to_float_kernel<<<64, 256, 0, st>>>(t->rate64, t->rate32, nr);
    split_float_kernel<<<256, 256, 0, st>>>(t->icdf64, t->icdf32, t->icdf32lo, ni);
    amm_table_kernel<<<d.n_chi, 256, 0, st>>>(d, t->amm64, t->amm32);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        free_tables(t);
        return QED_ERR_CUDA;
    }
    t->magic = kTablesMagic;
    *out = t;
    return QED_OK;
}

extern "C" qed_status qed_tables_export(qed_tables_t t, double* nlc_rate, double* nbw_rate, double* nlc_icdf,
                                        double* nbw_icdf) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    const size_t nc = t->desc.n_chi, ni = 2 * nc * t->desc.n_r;
    cudaError_t e = cudaSuccess;
    if (nlc_rate && e == cudaSuccess) e = cudaMemcpy(nlc_rate, t->rate64, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost);
    if (nbw_rate && e == cudaSuccess) e = cudaMemcpy(nbw_rate, t->rate64 + 2 * nc, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost);
    if (nlc_icdf && e == cudaSuccess) e = cudaMemcpy(nlc_icdf, t->icdf64, ni * sizeof(double), cudaMemcpyDeviceToHost);
    if (nbw_icdf && e == cudaSuccess) e = cudaMemcpy(nbw_icdf, t->icdf64 + ni, ni * sizeof(double), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_tables_export_amm(qed_tables_t t, double* ln_a) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    if (!ln_a) return QED_ERR_ARG;
    return cudaMemcpy(ln_a, t->amm64, t->desc.n_chi * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess
               ? QED_OK
               : QED_ERR_CUDA;
}

extern "C" qed_status qed_tables_destroy(qed_tables_t t) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    cudaDeviceSynchronize();
    free_tables(t);
    return QED_OK;
}

// ------------------------------------------------------------------------------------------------
// test entry points: the special functions and lookups exactly as the step kernels evaluate them
// ------------------------------------------------------------------------------------------------
namespace qed {
__global__ void bessel_eval_kernel(const double* bes64, const float* bes32, int prec, const double* x, double* out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (prec == QED_FP64) {
            double o[3];
            bessel64(bes64, x[i], o);
            for (int f = 0; f < 3; ++f) out[3 * i + f] = o[f];
        } else {
            float o[3];
            bessel32(bes32, (float)x[i], o);
            for (int f = 0; f < 3; ++f) out[3 * i + f] = o[f];
        }
    }
}

template <class R>
__global__ void lookup_kernel(TabP<R> T, const double* chi, const double* r, double* out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R c = (R)chi[i];
        const R lc = log_(c);
        R Iu, Id, Jp, Jm;
        nlc_rates(T, c, lc, Iu, Id);
        nbw_rates(T, c, lc, Jp, Jm);
        const R rr = (R)r[i];
        const R y = log_(rr) - log_(R(1) - rr);
        double* o = out + QED_LOOKUP_COLS * i;
        o[0] = Iu;
        o[1] = Id;
        o[2] = Jp;
        o[3] = Jm;
        o[4] = icdf_lookup(T, false, 0, lc, y);
        o[5] = icdf_lookup(T, false, 1, lc, y);
        o[6] = icdf_lookup(T, true, 0, lc, y);
        o[7] = icdf_lookup(T, true, 1, lc, y);
        o[8] = amm_lookup(T, c);
    }
}
}  // namespace qed

extern "C" qed_status qed_bessel_eval(qed_tables_t t, int32_t precision, const double* x, double* out, int64_t n,
                                      void* stream) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    if ((precision != QED_FP64 && precision != QED_FP32) || n < 0 || (n > 0 && (!x || !out))) return QED_ERR_ARG;
    if (n == 0) return QED_OK;
    bessel_eval_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(
        t->bes64, t->bes32, precision, x, out, n);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_tables_lookup(qed_tables_t t, int32_t precision, const double* chi, const double* r,
                                        double* out, int64_t n, void* stream) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    if ((precision != QED_FP64 && precision != QED_FP32) || n < 0 || (n > 0 && (!chi || !r || !out))) return QED_ERR_ARG;
    if (n == 0) return QED_OK;
    const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    if (precision == QED_FP64)
        lookup_kernel<double><<<g, 256, 0, (cudaStream_t)stream>>>(tab_params<double>(t), chi, r, out, n);
    else
        lookup_kernel<float><<<g, 256, 0, (cudaStream_t)stream>>>(tab_params<float>(t), chi, r, out, n);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}
