// qed_step32.cu -- FP32 fast path (placeholder until the FP32 kernels land).
#include "qed_steps.h"
void launch_lepton32(const qed_tables_s*, const qed_field&, const qed_step_desc&, const qed_particles*,
                     const qed_particles*, qed_counters*, cudaStream_t) {}
void launch_photon32(const qed_tables_s*, const qed_field&, const qed_step_desc&, const qed_particles*,
                     const qed_particles*, const qed_particles*, qed_counters*, cudaStream_t) {}
