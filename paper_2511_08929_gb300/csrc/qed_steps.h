// qed_steps.h -- per-step launch parameters and the launchers of the step kernels.
#pragma once
#include "qed_internal.h"

namespace qed {

struct StepP {
    double dt;
    double ph_hi;            // t + phase (FP64 path)
    float ph_hi_f, ph_lo_f;  // t + phase split into two floats (FP32 path): hi + lo
    float dt_f;
    uint32_t flags;
    uint64_t step, seed;
    double store_min, chi_floor;
    float store_min_f, chi_floor_f;  // the same thresholds rounded to float (FP32 path)
};

inline StepP step_params(const qed_step_desc& s, const qed_field& f) {
    StepP p;
    p.dt = s.dt;
    p.ph_hi = s.t + f.phase;
    p.ph_hi_f = (float)p.ph_hi;
    p.ph_lo_f = (float)(p.ph_hi - (double)p.ph_hi_f);
    p.dt_f = (float)s.dt;
    p.flags = s.flags;
    p.step = s.step;
    p.seed = s.seed;
    p.store_min = s.photon_store_min;
    p.chi_floor = s.chi_floor;
    p.store_min_f = (float)s.photon_store_min;
    p.chi_floor_f = (float)s.chi_floor;
    return p;
}

}  // namespace qed

void launch_lepton64(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* L,
                     const qed_particles* G, qed_counters* ctr, cudaStream_t st);
void launch_photon64(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* G,
                     const qed_particles* El, const qed_particles* Po, qed_counters* ctr, cudaStream_t st);
void launch_lepton32(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* L,
                     const qed_particles* G, qed_counters* ctr, cudaStream_t st);
void launch_photon32(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* G,
                     const qed_particles* El, const qed_particles* Po, qed_counters* ctr, cudaStream_t st);
