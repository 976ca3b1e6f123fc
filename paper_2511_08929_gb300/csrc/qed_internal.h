// qed_internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/qed.h"
#include "qed_bessel.cuh"

constexpr uint32_t kTablesMagic = 0x51454454u;  // "QEDT"

struct qed_tables_s {
    uint32_t magic;
    int device;
    qed_table_desc desc;
    double* rate64;  // [4][n_chi]: NLC up, NLC down, NBW +, NBW -
    double* icdf64;  // [4][n_chi][n_r]
    float* rate32;
    float* icdf32;
    float* icdf32lo;  // icdf64 - icdf32 rounded to float: the two floats hold an ICDF entry to ~1e-14
    double* bes64;  // [3][kBesN] scaled Bessel values
    float* bes32;
    double* amm64;  // [n_chi] ln a(chi_i), the field-dependent anomalous moment
    float* amm32;
};

inline bool valid_tables(const qed_tables_s* t) { return t != nullptr && t->magic == kTablesMagic; }

template <class R>
inline qed::TabP<R> tab_params(const qed_tables_s* t) {
    const R* rate = nullptr;
    const R* icdf = nullptr;
    if constexpr (sizeof(R) == 8) {
        rate = reinterpret_cast<const R*>(t->rate64);
        icdf = reinterpret_cast<const R*>(t->icdf64);
    } else {
        rate = reinterpret_cast<const R*>(t->rate32);
        icdf = reinterpret_cast<const R*>(t->icdf32);
    }
    const qed_table_desc& d = t->desc;
    qed::TabP<R> p;
    const size_t nc = d.n_chi;
    p.nlc_rate = rate;
    p.nbw_rate = rate + 2 * nc;
    p.nlc_icdf = icdf;
    p.nbw_icdf = icdf + 2 * nc * d.n_r;
    p.nlc_icdf_lo = nullptr;
    if constexpr (sizeof(R) == 4) p.nlc_icdf_lo = reinterpret_cast<const R*>(t->icdf32lo);
    if constexpr (sizeof(R) == 8) p.amm = reinterpret_cast<const R*>(t->amm64);
    else p.amm = reinterpret_cast<const R*>(t->amm32);
    const double dl = (std::log(d.chi_max) - std::log(d.chi_min)) / (d.n_chi - 1);
    p.lnchi_min = (R)std::log(d.chi_min);
    p.inv_dlnchi = (R)(1.0 / dl);
    p.chi_min = (R)d.chi_min;
    p.chi_max = (R)d.chi_max;
    p.y_lo = (R)d.y_lo;
    p.inv_dy = (R)((d.n_r - 1) / (d.y_hi - d.y_lo));
    p.inv_dy_lo = (R)((d.n_r - 1) / (d.y_hi - d.y_lo) - (double)p.inv_dy);
    p.n_chi = d.n_chi;
    p.n_r = d.n_r;
    return p;
}

// device view of one particle buffer
struct PartDev {
    double *x, *y, *z, *px, *py, *pz, *sx, *sy, *sz, *tau, *w;
    float4 *q0, *q1, *q2;
    uint64_t* id;
    int64_t* count;
    int64_t* begin;  // number of particles a step processes (NULL: *count at launch)
    int64_t* dead;
    int64_t* n_dead;
    int64_t capacity;
};

inline PartDev part_dev(const qed_particles* p) {
    PartDev d;
    d.x = p->x; d.y = p->y; d.z = p->z;
    d.px = p->px; d.py = p->py; d.pz = p->pz;
    d.sx = p->sx; d.sy = p->sy; d.sz = p->sz;
    d.tau = p->tau; d.w = p->w;
    d.q0 = reinterpret_cast<float4*>(p->q0);
    d.q1 = reinterpret_cast<float4*>(p->q1);
    d.q2 = reinterpret_cast<float4*>(p->q2);
    d.id = p->id;
    d.count = p->count;
    d.begin = p->begin;
    d.dead = p->dead;
    d.n_dead = p->n_dead;
    d.capacity = p->capacity;
    return d;
}

// the reservation state of a step call: the append_* fields at the end of the caller's counters
__host__ __device__ inline qed::AppendState* append_state(qed_counters* ctr) {
    return reinterpret_cast<qed::AppendState*>(&ctr->append_base[0]);
}

// the switches a step accepts: every flag of the header, without the contradictory anomalous-moment
// pairs (a(chi) in T-BMT and the loop's Scorer term are the same moment; g = 2 excludes both)
inline bool valid_flags(uint32_t f) {
    const uint32_t known =
        QED_F_FULL | QED_F_TBMT_PAPER | QED_F_AMM | QED_F_LOOP | QED_F_G2 | QED_F_BETA_BASIS | QED_F_REJECT;
    if (f & ~known) return false;
    return !((f & QED_F_AMM) && (f & (QED_F_LOOP | QED_F_G2)));
}

// validation of a particle buffer for a given layout
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline qed_status check_particles(const qed_particles* p, bool need_dead) {
    if (!p || !p->count || !p->id || p->capacity < 0) return QED_ERR_ARG;
    if (p->layout == QED_FP64) {
        if (!p->x || !p->y || !p->z || !p->px || !p->py || !p->pz || !p->sx || !p->sy || !p->sz || !p->tau || !p->w)
            return QED_ERR_ARG;
    } else if (p->layout == QED_FP32) {
        if (!p->q0 || !p->q1 || !p->q2 || !aligned16(p->q0) || !aligned16(p->q1) || !aligned16(p->q2)) return QED_ERR_ARG;
    } else {
        return QED_ERR_ARG;
    }
    if (need_dead && (!p->dead || !p->n_dead)) return QED_ERR_ARG;
    return QED_OK;
}

template <class R>
inline qed::FieldP<R> field_params(const qed_field& f) {
    qed::FieldP<R> p;
    p.kind = f.kind;
    p.a0 = (R)f.a0;
    p.inv2n = (R)(f.n_cycles > 0 ? 0.5 / f.n_cycles : 0.0);
    p.phimax = (R)(2.0 * qed::kPi * f.n_cycles);
    p.E0x = (R)f.E0[0]; p.E0y = (R)f.E0[1]; p.E0z = (R)f.E0[2];
    p.B0x = (R)f.B0[0]; p.B0y = (R)f.B0[1]; p.B0z = (R)f.B0[2];
    p.eta0 = (R)f.eta0;
    return p;
}

inline bool valid_field(const qed_field* f) {
    return f && f->kind >= QED_FIELD_CONST && f->kind <= QED_FIELD_ROT_B && std::isfinite(f->a0) &&
           std::isfinite(f->phase) && f->eta0 > 0.0 && std::isfinite(f->eta0) &&
           (f->kind == QED_FIELD_CONST || f->n_cycles > 0.0);
}

inline int launch_blocks(int64_t work, int threads) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int64_t need = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
}

// The learned sampler inside the batched step (defined with the network in qed_mlp.cu): the network's
// validity check, the persistent grid of its sampling kernel for up to n_max samples, and that kernel
// over the first min(n_max, *n_dev) samples (n_dev a count on the device, written by an earlier kernel
// of the same stream), checked at tol with the tables' mixture quantile as fallback.
bool mlp_valid(qed_mlp_t m);
int mlp_listed_grid(int64_t n_max);
qed_status mlp_sample_listed(qed_mlp_t m, const qed_tables_s* t, const double* chi, const double* r, const double* s,
                             int64_t n_max, const unsigned long long* n_dev, double tol, float* out4,
                             unsigned long long* n_fallback, int grid, cudaStream_t st);
