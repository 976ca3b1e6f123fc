/*
 * qed.h -- C ABI of libqedgb, a GB300 (sm_103a) implementation of the per-particle,
 * per-time-step spin- and polarization-resolved strong-field QED step of
 * Qian, Seipt, Vranic, Grismayer, Ridgers and Thomas, "A Fully Spin and
 * Polarization Resolved Strong Field QED Algorithm for Particle-in-Cell Codes"
 * (arXiv:2511.08929).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units: time 1/omega, length c/omega, momentum m c, fields m c omega / e,
 *    photon energy m c^2.  eta0 = hbar omega / (m c^2); the Schwinger field is 1/eta0.
 *  - Pointers named *_dev, and every array reached through qed_particles and
 *    qed_counters, are DEVICE pointers (cudaMalloc / PyTorch CUDA tensors) owned by
 *    the caller.  Pointers named host_* are host memory owned by the caller.  The
 *    table handle owns its device memory and is freed by qed_tables_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call only enqueues work on it and returns, except where "synchronizes"
 *    is written.  Calls are graph-capturable unless stated otherwise: particle
 *    counts live in device memory and are read and updated by the kernels.
 *  - Argument errors are returned synchronously (QED_ERR_ARG) and nothing is
 *    enqueued.  Errors found on the device (capacity exhausted, non-finite input,
 *    chi beyond the table) never trap: they are counted in qed_counters and the
 *    first one sets qed_counters.status / first_bad, read back by qed_counters_read.
 *  - All random numbers are Philox4x32-10 (Salmon et al., SC'11) keyed by
 *    key = id ^ seed, counter = (step_lo, step_hi, slot, 0), so results do not
 *    depend on launch configuration, and daughters get ids from the same stream.
 *  - Thread safety: calls on different streams may run concurrently when they touch
 *    disjoint particle buffers and counters; the table handle is read-only after build.
 */
#ifndef QED_H
#define QED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QED_ABI_VERSION 3

typedef enum {
    QED_OK = 0,
    QED_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, misaligned buffer) */
    QED_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    QED_ERR_CAPACITY = -3, /* device: a daughter did not fit in its buffer (counted, not applied) */
    QED_ERR_RANGE = -4,    /* device: chi above the table range (clamped and counted) */
    QED_ERR_NAN = -5,      /* device: a particle with non-finite state was skipped */
    QED_ERR_TIMEOUT = -6,  /* device: a bounded wait gave up */
    QED_ERR_STATE = -7,    /* handle used after destroy, or library not initialised */
    QED_ERR_NOMEM = -8,    /* device allocation failed */
    QED_ERR_TOO_LARGE = -9 /* a size above the fixed limit of the call (qed_compact_noalloc) */
} qed_status;

/* Particle buffer layouts = the two arithmetic paths. */
enum {
    QED_FP64 = 0, /* plain path: eleven double planes, all arithmetic in FP64 */
    QED_FP32 = 1  /* fast path: three float4 planes; push, rates and sampling in FP32,
                     optical depth and spin renormalisation in FP64 */
};

/* Species charge (qed_particles.charge). */
enum { QED_ELECTRON = -1, QED_PHOTON = 0, QED_POSITRON = 1 };

/* Physics switches (qed_step_desc.flags); the paper's "flexible switch" of Sec. 8.5.1. */
enum {
    QED_F_TAU = 1u << 0,           /* optical-depth event decision (Sec. 4.1); else r1 < W dt per step */
    QED_F_RECOIL = 1u << 1,        /* radiation reaction p_f = (1 - lambda) p_i (Sec. 5.1) */
    QED_F_SPIN_COLLAPSE = 1u << 2, /* s_f = +-S_SQA (Sec. 5.1, 5.2); else the expectation value */
    QED_F_POL_COLLAPSE = 1u << 3,  /* xi = +-Xi_PQA (Sec. 5.1); else xi = F/F0 */
    QED_F_NONTRANSITION = 1u << 4, /* spin / polarization update without an event (Sec. 6) */
    QED_F_PUSH = 1u << 5,          /* Boris momentum push */
    QED_F_TBMT = 1u << 6,          /* T-BMT spin precession (Sec. 8.3) */
    QED_F_TBMT_PAPER = 1u << 7,    /* T-BMT v x E coefficient as printed, (a + 1/gamma) */
    QED_F_EMIT = 1u << 8,          /* QED events: NLC for leptons, NBW for photons */
    QED_F_RESOLVED = 1u << 9,      /* rates and sampling depend on s.beta / xi3 (Sec. 5.1, 5.2) */
    QED_F_MOVE = 1u << 10,         /* position advance */
    QED_F_SPIN_EVENT = 1u << 11,   /* lepton spin changes at emission; pair daughters get spins */
    QED_F_POL_EVENT = 1u << 12,    /* emitted photons carry the Stokes vector of F (else unpolarized) */
    /* The anomalous moment in the spin precession (Sec. 8.6.2, App. A.1 one-loop terms).  Default: the
     * zero-field a = alpha/(2 pi) in T-BMT.  QED_F_AMM: T-BMT with the field-dependent a(chi) of the loop's
     * Scorer term, chi taken at the time-centred momentum.  QED_F_LOOP: T-BMT with g = 2, and the loop's
     * Scorer term applied in the no-emission update instead (a turn about the rest-frame magnetic field
     * by a(chi) chi dt / (eta0 gamma); needs QED_F_EMIT).  QED_F_G2: T-BMT with g = 2 and no loop term
     * (the paper's g = 2 comparison).  QED_F_AMM with QED_F_LOOP or QED_F_G2 is QED_ERR_ARG. */
    QED_F_AMM = 1u << 13,
    QED_F_LOOP = 1u << 14,
    QED_F_G2 = 1u << 15,
    /* Spins resolved along +-beta (the rest-frame magnetic direction) instead of the spin quantization
     * axis (Sec. 8.3 compares the two): an emitting lepton ends at -beta with probability
     * (w - g.beta)/(2w), else +beta (expectation mode: (g.beta/w) beta); pair daughters take the four
     * states along (+-beta, +-beta) with probabilities G_ab/(4 w0) (expectation: (j.beta/w0) beta). */
    QED_F_BETA_BASIS = 1u << 16,
    /* Table-free decision and sampling by rejection (Sec. 4.2): per step a candidate energy fraction
     * lambda = r1^3 (emission; the f = r^3 proposal) or lambda = r1 (pair, positron fraction) is accepted
     * if r2 < 3 r1^2 (dW/dlambda) dt (emission) or r2 < (dW/dlambda) dt (pair), with dW/dlambda the
     * spin- (polarization-) resolved density of App. A; the ICDF tables and the optical depth are not
     * used (the 1-D rate tables still serve the no-emission update).  Steps whose acceptance exceeds 1
     * (dt too long for the method) are counted in bound_exceeded. */
    QED_F_REJECT = 1u << 17
};
#define QED_F_FULL                                                                                     \
    (QED_F_TAU | QED_F_RECOIL | QED_F_SPIN_COLLAPSE | QED_F_POL_COLLAPSE | QED_F_NONTRANSITION |       \
     QED_F_PUSH | QED_F_TBMT | QED_F_EMIT | QED_F_RESOLVED | QED_F_MOVE | QED_F_SPIN_EVENT | QED_F_POL_EVENT)

/* Analytic fields that stand in for the PIC grid fields (Sec. 4). */
enum {
    QED_FIELD_CONST = 0,     /* E = E0, B = B0 */
    QED_FIELD_LP = 1,        /* E = a0 g(phi) cos(phi) x, B = z x E, phi = t - z + phase */
    QED_FIELD_CP = 2,        /* E = a0 g(phi) (cos phi, sin phi, 0), B = z x E */
    QED_FIELD_CP_COUNTER = 3, /* CP plus a CP wave along -z with phi2 = t + z + phase, B2 = -z x E2 */
    QED_FIELD_ROT_B = 4       /* E = 0, B = B0[2] (0, sin th, cos th), th = (pi/2) clamp((t + phase) /
                                 (2 pi n_cycles), 0, 1): a uniform field turning from z to y (the
                                 rotating-field test of Sec. 8.3) */
};

typedef struct {
    int32_t kind;
    int32_t pad;
    double a0;       /* peak amplitude per component, units of m c omega / e */
    double n_cycles; /* envelope g = sin^2(phi / (2 n_cycles)) on 0 <= phi <= 2 pi n_cycles, else 0 */
    double phase;    /* added to t - z (and to t + z for the counter-propagating wave) */
    double E0[3], B0[3];
    double eta0;     /* hbar omega / (m c^2) of the laser that sets the units */
} qed_field;

/* Rate and inverse-CDF tables (Sec. 5.1: W_up/W_down and IntF^-1_up/down;
 * Sec. 5.2: W_+/W_- and IntG^-1_+/-).
 *   chi_i = exp(ln chi_min + i dlnchi), i < n_chi; y_m = y_lo + m dy, m < n_r, r_m = 1/(1 + e^-y_m).
 *   NLC rate  ln I_s(chi_i),  I_s = int_0^1 [-IntK13(u') + kappa K23(u') + s lambda K13(u')] d lambda
 *   NBW rate  ln(J_s(chi_i) e^{8/(3 chi_i)}),  J_s = int_0^1 [IntK13 + rho K23 - s K23](u~') d lambda
 *   NLC ICDF  ln u'(chi_i, r_m),  the u' = 2 lambda / (3 chi (1 - lambda)) below which a fraction r_m
 *             of the spectrum lies
 *   NBW ICDF  ln x(chi_i, r_m),   x = u~' - 8/(3 chi) of the spectrum folded about lambda = 1/2,
 *             counted from the centre
 * Lookups interpolate linearly in (ln chi, value) between rows and by 4-point Lagrange in y along a row;
 * below y_lo the asymptote (u' ~ r^3, x ~ r^2), above y_hi the last entry. */
typedef struct {
    double chi_min, chi_max;
    int32_t n_chi; /* >= 2 */
    int32_t n_r;   /* >= 4 */
    double y_lo, y_hi;
} qed_table_desc;

typedef struct qed_tables_s *qed_tables_t;

/* One particle species in structure-of-arrays form.  For photons, (px, py, pz) is the
 * momentum hbar k and (sx, sy, sz) the polarization vector P of Sec. 3.2.
 *   layout QED_FP64: x..w are eleven double arrays of `capacity` entries.
 *   layout QED_FP32: three float4 arrays of `capacity` entries (16-byte aligned); tau is the FP64 optical
 *                    depth stored as the low and high 32-bit words of its bit pattern.
 *                    leptons: q0 = (x, y, z, px), q1 = (py, pz, sx, sy), q2 = (sz, w, tau_lo, tau_hi);
 *                    photons: q0 = (x, y, z, sx), q1 = (sy, sz, tau_lo, tau_hi), q2 = (px, py, pz, w)
 *                    (a photon step never changes k or w: it rewrites q0 and q1, or q0 alone when the
 *                    photon has no pair rate).
 * id: uint64 array; the Philox key of each particle.  count: device int64, the live count, advanced
 * by the kernels that append daughters.  begin: optional device int64; when set, a step call processes
 * particles [0, *begin) instead of [0, *count at launch), so that daughters appended during the current
 * step by another call are not stepped until the next one (qed_snapshot_counts sets it).
 * dead / n_dead (photons only): device list of the indices that converted to pairs, consumed by
 * qed_compact; converted photons keep momentum 0 and weight 0 until then. */
typedef struct {
    int32_t layout;
    int32_t charge;
    int64_t capacity;
    int64_t *count;
    int64_t *begin;
    double *x, *y, *z, *px, *py, *pz, *sx, *sy, *sz, *tau, *w;
    float *q0, *q1, *q2;
    uint64_t *id;
    int64_t *dead;
    int64_t *n_dead;
} qed_particles;

/* Per-step parameters. */
typedef struct {
    double dt;        /* step length */
    double t;         /* time at the start of the step (fields are taken at t and the pre-push position) */
    uint64_t step;    /* step index: the Philox counter */
    uint64_t seed;    /* xored into the Philox key */
    uint32_t flags;   /* QED_F_* */
    uint32_t pad;
    double photon_store_min; /* emitted photons with |k| below this are not stored (Sec. 4.2); 0 keeps all */
    double chi_floor;        /* no QED event is considered below this chi */
} qed_step_desc;

/* Device-resident counters, accumulated by every step call (zero them with cudaMemset).
 *
 * Buffer overflow.  A step call takes the counts of its daughter buffers when it begins and appends
 * at most what fits: an event whose daughters do not all fit is not applied (the parent keeps the state
 * the classical part of its step gave it, its optical depth stays spent, so it tries again next step)
 * and is counted in dropped_capacity, status QED_ERR_CAPACITY.  An electron-positron pair is stored
 * whole or not at all.  Which events of an overflowing call get the last free slots is not specified
 * (the reservation order of the device); counts never exceed capacity. */
typedef struct {
    unsigned long long events;           /* emissions (push step) or pair conversions (pair step) */
    unsigned long long stored;           /* daughters written */
    unsigned long long dropped_capacity; /* daughters that did not fit */
    unsigned long long chi_clamped;      /* particle-steps with chi above chi_max */
    unsigned long long renormalised;     /* spin / Stokes vectors rescaled to unit length */
    unsigned long long below_store;      /* photons not stored because |k| < photon_store_min */
    unsigned long long nonfinite;        /* particles skipped because their state was not finite */
    unsigned long long rate_steps;       /* FP32 paths: photon-steps with a nonzero pair rate (the others
                                            only move, and write the position plane alone) */
    unsigned long long bound_exceeded;   /* QED_F_REJECT: particle-steps whose acceptance exceeded 1 */
    int32_t status;                      /* first device-side error (qed_status), 0 if none */
    int32_t pad;
    int64_t first_bad;                   /* particle index of the first device-side error, -1 if none */
    /* Daughter-slot reservation of the step call in flight, written only by that call's own kernels:
     * the daughter buffers' counts when the call began, how many events' daughters fit, how many
     * events asked for slots.  Callers neither read nor set it (zeroing it with the rest is fine); it
     * is the reason calls that share one qed_counters must not overlap on the device. */
    int64_t append_base[2];
    int64_t append_budget;
    unsigned long long append_next;
} qed_counters;

/* ---------------------------------------------------------------------------------------------- */

/* Version of this header the library was built from. */
int32_t qed_abi_version(void);

/* Human-readable name of a status code (static storage). */
const char *qed_status_string(int32_t status);

/* Build the FP64 tables on the current device (Sec. 5.1 and 5.2 rate and ICDF tables, from the
 * Bessel-function forms of App. A).  All integrals are evaluated in FP64 to full precision; the FP32
 * path uses a float copy made here too.  Synchronizes `stream` before returning.
 * Errors: QED_ERR_ARG (bad desc or null out), QED_ERR_NOMEM, QED_ERR_CUDA. */
qed_status qed_tables_build(const qed_table_desc *desc, qed_tables_t *out, void *stream);

/* Copy the FP64 tables to host arrays: rates [2][n_chi] (index 0 = up / xi3 = +1, 1 = down / xi3 = -1),
 * ICDFs [2][n_chi][n_r].  Any pointer may be NULL to skip it.  Synchronous. */
qed_status qed_tables_export(qed_tables_t t, double *host_nlc_rate, double *host_nbw_rate, double *host_nlc_icdf,
                             double *host_nbw_icdf);

/* Copy the table of the field-dependent anomalous moment to the host: ln a(chi_i) on the rate grid,
 * double[n_chi] (one-loop Scorer term of App. A.1, a(chi) = (alpha/chi) int_0^1 dlambda lambda Gi(z)/sqrt(z),
 * z = (lambda/(chi (1 - lambda)))^{2/3}, built in FP64 with the other tables).  Synchronous. */
qed_status qed_tables_export_amm(qed_tables_t t, double *host_ln_a);

/* Free the tables.  Synchronizes the device. */
qed_status qed_tables_destroy(qed_tables_t t);

/* Evaluate the device implementations of e^x K_{1/3}(x), e^x K_{2/3}(x), e^x int_x^inf K_{1/3} (App. A
 * Bessel forms) for n arguments: precision QED_FP64 (table + series, FP64) or QED_FP32 (float table).
 * x_dev: double[n]; out_dev: double[3 n] (k13, k23, intk13 interleaved).  For tests of the special
 * functions used by the step kernels. */
qed_status qed_bessel_eval(qed_tables_t t, int32_t precision, const double *x_dev, double *out_dev, int64_t n,
                           void *stream);

/* Look up the tables for n values of chi and r exactly as the step kernels do (FP64 or FP32 arithmetic):
 * out_dev: double[6 n] = (I_up, I_down, ln u'_up(r), ln u'_down(r), J_+ e^{..}..) -- see qed_lookup_layout
 * below.  For tests of the interpolation rules. */
qed_status qed_tables_lookup(qed_tables_t t, int32_t precision, const double *chi_dev, const double *r_dev,
                             double *out_dev, int64_t n, void *stream);
/* out_dev row layout of qed_tables_lookup: [0] I_up(chi), [1] I_down(chi), [2] J_+(chi), [3] J_-(chi)
 * (unscaled), [4] ln u' from the up ICDF, [5] ln u' from the down ICDF, [6] ln x from the + ICDF,
 * [7] ln x from the - ICDF (NBW rows take r as the folded coordinate), [8] a(chi), the field-dependent
 * anomalous moment (linear in (ln chi, ln a) between nodes, the end values outside the grid). */
#define QED_LOOKUP_COLS 9

/* Optical depth at birth for particles [begin, *count): tau = -ln u(id, step = 2^64 - 1, slot 0)
 * (Sec. 4.1, optical-depth method). */
qed_status qed_init_tau(qed_particles *p, uint64_t seed, int64_t begin, void *stream);

/* One lepton step (Sec. 5.1 and its flow chart; Sec. 6 non-emission update): for every lepton in
 * [0, *count at launch): fields at (x, t), Boris push, T-BMT precession, position advance, chi and the
 * (eps, beta, k) basis, W_s, optical depth; on emission lambda from the ICDF, recoil, SQA collapse of
 * the spin, PQA collapse of the photon Stokes vector, and a photon appended to `photons` (its P vector
 * in the emission basis); without emission the non-emission spin update.  leptons->charge must be
 * QED_ELECTRON or QED_POSITRON.  Photons appended this step are not stepped until the next call.
 * photons may be NULL (emitted photons are then counted as dropped).  leptons and photons must have the
 * same layout.  counters_dev: device qed_counters (accumulated). */
qed_status qed_push_step(qed_tables_t t, const qed_field *field, const qed_step_desc *step, qed_particles *leptons,
                         qed_particles *photons, qed_counters *counters_dev, void *stream);

/* One photon step (Sec. 5.2 and its flow chart; Sec. 6 non-pair update): ballistic move, chi_gamma,
 * basis, Stokes from P, W_xi, optical depth; on conversion lambda from the folded ICDF, the four
 * correlated spin states of the pair, an electron and a positron appended (both at the photon's
 * position), and the photon flagged dead (appended to photons->dead); otherwise the non-pair update of
 * the Stokes vector.  A pair that does not fit leaves the photon alive (it retries next step). */
qed_status qed_pair_step(qed_tables_t t, const qed_field *field, const qed_step_desc *step, qed_particles *photons,
                         qed_particles *electrons, qed_particles *positrons, qed_counters *counters_dev,
                         void *stream);

/* Remove the photons listed in photons->dead (Sec. 4.3: converted photons leave the simulation) by
 * moving live photons from the tail into the holes; the order of the survivors changes, their set does
 * not.  Resets *n_dead to 0.  workspace: device memory of at least qed_compact_workspace_bytes(capacity)
 * bytes (16-byte aligned), owned by the caller, zeroed (cudaMemset) before its first use; every call
 * leaves it ready for the next one.  Calls that share a workspace must not overlap on the device. */
qed_status qed_compact(qed_particles *photons, void *workspace, size_t workspace_bytes, void *stream);
size_t qed_compact_workspace_bytes(int64_t capacity);

/* qed_compact without a workspace argument, and without any allocation (no cudaMalloc or cudaFree,
 * no allocating library).  The paper has no counterpart: this is bookkeeping of the library, for
 * callers that cannot allocate or hand over device memory at the call site -- host codes whose device
 * memory is handed out entirely by their own pool, and step loops that must stay asynchronous
 * (cudaFree, and cudaMalloc under memory pressure, synchronise the device).
 *
 * Scratch: a file-scope device array sized for QED_COMPACT_NOALLOC_MAX_CAPACITY photons (4.25 MiB
 * per device), zero at module load.  Each call resets the header counters in its first kernel and
 * clears, in its third, every tail mark its second set, so it leaves the scratch ready for the next call
 * and nothing has to be cleared by the caller; a call costs O(dead photons), like qed_compact.
 * Result: the same as qed_compact (the survivors' set; their order may differ).
 *
 * Limits and ordering:
 *  - photons->capacity above QED_COMPACT_NOALLOC_MAX_CAPACITY returns QED_ERR_TOO_LARGE before any
 *    device work; use qed_compact with a caller workspace there.
 *  - All calls on one device share the one scratch: calls that overlap on the device (streams with no
 *    ordering between them, or several host threads) race on it and corrupt the result.  Order them
 *    on one stream or with events.
 *  - The first call on each device looks the scratch up (cudaGetSymbolAddress with that device
 *    current, which may load the module); make that first call before any stream capture begins.
 *    The address is kept per device index for the life of the process: after cudaDeviceReset (or any
 *    teardown of the device's primary context) it is stale, so do not call this function again in that
 *    process once the device has been reset.
 * Errors: QED_ERR_ARG (bad buffer), QED_ERR_TOO_LARGE, QED_ERR_CUDA (lookup or launch failed). */
#define QED_COMPACT_NOALLOC_MAX_CAPACITY 262144
qed_status qed_compact_noalloc(qed_particles *photons, void *stream);

/* ---- Batched collisions: many independent instances stepped together ----
 * A batch is a set of independent collision instances (each its own laser, seed and three FP32 species
 * buffers) advanced in lockstep.  One time step of the whole batch is: a planning kernel (alive counts
 * at step start, the tile list over all instances and species, each one's step context), one
 * persistent kernel that streams every tile of 32 particles of every instance (the lepton step of
 * Sec. 5.1 for electrons and positrons, the photon step of Sec. 5.2 for photons, each as qed_push_step /
 * qed_pair_step do) and lists the particles whose optical depth ran out, an event kernel that runs the
 * emission / pair branch for the listed particles, and the photon compaction of every instance.  The step index and time live in device memory and advance on the
 * device, so a captured CUDA graph of one or more steps is replayed unchanged.  Results are the ones
 * qed_push_step, qed_pair_step and qed_compact give per instance with begin snapshots (the same
 * arithmetic and random draws; appended daughters may sit in another order), whatever the tuning. */
#define QED_BATCH_MAX_INSTANCES 1024
#define QED_BATCH_VARIANTS 5

typedef struct qed_batch_s *qed_batch_t;

typedef struct {
    qed_field field; /* the instance's laser */
    uint64_t seed;   /* the instance's Philox seed */
    qed_particles electrons, positrons, photons; /* layout QED_FP32; photons with a dead list; begin unused */
} qed_instance;

typedef struct {
    double dt;       /* time step of every instance */
    double t0;       /* time of step step0; step k is at t0 + (k - step0) dt (rounded as a product, then a sum) */
    uint64_t step0;  /* Philox step index of the first step */
    uint32_t flags;  /* QED_F_* */
    int32_t pad;
    double photon_store_min, chi_floor; /* as in qed_step_desc */
} qed_batch_desc;

/* Launch shape of the batch step (no effect on results).
 *   variant       kernel build (threads per block, tiles of 32 particles in flight per warp, registers
 *                 sized for so many blocks per SM): 0 = 256, 3, 3; 1 = 256, 3, 2; 2 = 256, 2, 4;
 *                 3 = 512, 2, 1; 4 = 512, 2, 2
 *   blocks_per_sm resident blocks per SM of the persistent grid (0: the occupancy maximum)
 *   chunk         the most consecutive tiles of 32 particles a warp takes from the step's work counter at
 *                 once (takes shrink towards 2 as the step's work runs out)
 *   graph_steps   time steps captured per CUDA graph (0: launch the kernels directly every step) */
typedef struct {
    int32_t variant, blocks_per_sm, chunk, graph_steps;
} qed_batch_tuning;

typedef struct {
    uint64_t step;              /* Philox index of the next step */
    uint64_t particle_steps;    /* particles processed since creation (all instances and species) */
    uint64_t species_steps[3];  /* the same split into electrons, positrons, photons */
    int64_t alive[3];           /* electrons, positrons, photons processed by the last step */
} qed_batch_stats;

/* Create a batch of n_inst (1 .. QED_BATCH_MAX_INSTANCES) instances.  The instance array is copied; the
 * particle buffers stay the caller's and must outlive the batch.  The batch owns its device planning
 * state, the compaction workspace (17 B per photon of capacity) and the step's event list (8 B per
 * particle of capacity), and writes its counters to counters_dev.  Errors: QED_ERR_ARG, QED_ERR_STATE (tables), QED_ERR_NOMEM, QED_ERR_CUDA. */
qed_status qed_batch_create(qed_tables_t t, const qed_instance *instances, int32_t n_inst, const qed_batch_desc *desc,
                            qed_counters *counters_dev, qed_batch_t *out);
/* Set / read the launch shape; setting it discards any captured graph. */
qed_status qed_batch_set_tuning(qed_batch_t b, const qed_batch_tuning *tuning);
qed_status qed_batch_get_tuning(qed_batch_t b, qed_batch_tuning *out);
/* Advance every instance n_steps time steps on `stream` (asynchronous).  With graph_steps > 0 the steps
 * run as launches of a CUDA graph of graph_steps steps, captured on first use; the rest directly.
 * n_steps = 0 only captures the graph (if graph_steps > 0 and none is held), so that the capture and
 * instantiation can be kept out of a timed region. */
qed_status qed_batch_step(qed_batch_t b, int32_t n_steps, void *stream);
/* Kernel timing: events[2k], events[2k+1] (cudaEvent_t, created by the caller with timing enabled) are
 * recorded before the persistent kernel and after the event kernel of the k-th step (k modulo n_pairs)
 * of every CUDA graph captured from now on (step k of the graph) and of directly launched steps (counted
 * from this call).  n_pairs = 0 switches it off.  Discards any captured graph. */
qed_status qed_batch_set_kernel_events(qed_batch_t b, void *const *events, int32_t n_pairs);
/* Autotuner: times the persistent and event kernels of every launch shape it considers on the batch's
 * own next steps (they are real steps: results do not depend on the shape), picks the one with the least
 * time per particle-step and sets it.  steps_per_candidate >= 1.  cache_path (may be NULL): a text file of
 * one JSON object per line, keyed by device, SM count and workload size; a matching line is used
 * without timing, a new result is appended.  Synchronizes `stream`. */
qed_status qed_batch_tune(qed_batch_t b, int32_t steps_per_candidate, const char *cache_path, qed_batch_tuning *out,
                          void *stream);
/* Step index and processed particle-steps (synchronizes `stream`). */
qed_status qed_batch_stats_read(qed_batch_t b, qed_batch_stats *out, void *stream);
void qed_batch_destroy(qed_batch_t b);

/* ---- Learned sampler (no counterpart code in the paper; Sec. 5.1 rejects a direct table in
 * (chi, r, s_beta) for its memory, and this network stands in for it) ----
 * Network 3 -> 64 -> 64 -> 64 -> 4 with SiLU.  Inputs ((ln chi - m)/h over chi in [1e-3, 1e2],
 * clamp(logit r, +-20)/10, s_beta).  Outputs: 100 x the corrections to the rate-weighted blend of the two
 * spin-branch quantiles ln u'(chi, r) of the tables (and to xi3 there), and 100 xi1, 100 xi2.  Layer 1
 * runs in FP32; layers 2-4 take BF16-rounded weights and activations on tensor cores with FP32
 * accumulation.  Parameters: one FP32 array of QED_MLP_PARAMS = W1[64][3] b1[64] W2[64][64] b2[64]
 * W3[64][64] b3[64] W4[4][64] b4[4] (weights row = output unit). */
#define QED_MLP_PARAMS 8836
#define QED_MLP_ALWAYS_TABLE 1 /* qed_mlp_sample flag: skip the network (the table path, for comparison) */
/* qed_mlp_sample flag: instead of the network, the sampler the step's event pass runs (Sec. 5.1): the spin
 * branch chosen with probability W_down (1 - s)/(2 W_s), the uniform rescaled within it, one row of that
 * branch's ICDF (float-float), xi3 at the sampled u'; out4 = (ln u', 0, 0, xi3), no check, no fallback */
#define QED_MLP_BRANCH_TABLE 2

typedef struct qed_mlp_s *qed_mlp_t;

/* A network with the given initial parameters (host array of QED_MLP_PARAMS floats) and device scratch
 * for training batches of up to max_batch samples.  Errors: QED_ERR_ARG, QED_ERR_NOMEM, QED_ERR_CUDA. */
qed_status qed_mlp_create(int64_t max_batch, const float *init_params, qed_mlp_t *out);
void qed_mlp_destroy(qed_mlp_t m);
/* Copy the parameters to / from host memory (setting resets the optimiser state).  Synchronous. */
qed_status qed_mlp_get_params(qed_mlp_t m, float *host_out);
qed_status qed_mlp_set_params(qed_mlp_t m, const float *host_in);
/* Training samples from the FP64 tables: sample first_index + i draws chi (log-uniform over [1e-3, 1e2]),
 * r and s_beta (uniform) from Philox(id = first_index + i, seed, step 2^64 - 2, slots 0 and 1); x_dev gets
 * its n x 3 features, y_dev its n x 4 targets (the exact mixture quantile, found by regula falsi between
 * the branch quantiles on the mixture CDF of the interpolated branch rows, and xi3 there, minus the
 * blend baseline, times 100), raw_dev (may be NULL) n x 3 doubles (chi, r, s_beta). */
qed_status qed_mlp_targets(qed_tables_t t, int64_t n, uint64_t seed, int64_t first_index, float *x_dev, float *y_dev,
                           double *raw_dev, void *stream);
/* Forward and backward pass of one batch (n <= max_batch): grad_dev gets dL/dparameters for
 * L = mean over the batch of the squared error summed over the four outputs; loss_dev (may be NULL) L. */
qed_status qed_mlp_grad(qed_mlp_t m, const float *x_dev, const float *y_dev, int64_t n, float *grad_dev,
                        float *loss_dev, void *stream);
/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay on weights only). */
qed_status qed_mlp_adamw(qed_mlp_t m, const float *grad_dev, float lr, float weight_decay, void *stream);
/* steps x (fresh batch of targets at first_index + k batch, forward, backward, AdamW), learning rate
 * decaying from lr to lr_final on a cosine; loss_per_step_dev (may be NULL) gets each step's loss. */
qed_status qed_mlp_train(qed_mlp_t m, qed_tables_t t, int64_t steps, int64_t batch, uint64_t seed, int64_t first_index,
                         float lr, float lr_final, float weight_decay, float *loss_per_step_dev, void *stream);
/* Raw network outputs (n x 4) for feature rows x_dev (n x 3), on tensor cores. */
qed_status qed_mlp_forward(qed_mlp_t m, const float *x_dev, int64_t n, float *out_dev, void *stream);
/* The sampler: for device arrays chi, r, s_beta (n doubles each), out4 (n x 4 floats) = (ln u', xi1,
 * xi2, xi3) from the network, checked: the exact mixture CDF of the tables at ln u' must be within tol of
 * r and the Stokes vector within tol of its closed form there, else (or with QED_MLP_ALWAYS_TABLE) the
 * table path (the exact mixture quantile, the closed-form Stokes vector).  fell_back (n bytes,
 * may be NULL) marks the samples that took the table path; err_out (n floats, may be NULL) gets the
 * network's CDF error |C(ln u') - r| (-1 where the network was skipped); *n_fallback (device, may be
 * NULL) is incremented by the number of fallbacks. */
qed_status qed_mlp_sample(qed_mlp_t m, qed_tables_t t, const double *chi, const double *r, const double *s_beta,
                          int64_t n, double tol, int32_t flags, float *out4, uint8_t *fell_back, float *err_out,
                          unsigned long long *n_fallback, void *stream);

/* The learned sampler on the batched step's event path: with m set, the energy fraction of every
 * emission (NLC event) of each step comes from the network instead of the branch choice and ICDF row
 * (Sec. 5.1), checked on its quantile as qed_mlp_sample checks it (mixture CDF within tol of the
 * uniform r2, else the tables' mixture quantile).  Each step then runs, between the streaming pass and
 * the event pass, a kernel that gathers (chi, r2, s.beta) of the listed events and the sampler over
 * them.  The network's Stokes outputs are neither used nor checked (out4[1..3] are 0): the event
 * computes the photon's Stokes vector from the spectra at the sampled u' with the collapsed final spin,
 * which the network cannot know.  m = NULL restores the tables.  The batch keeps the pointer, not the
 * network: m must outlive its use.  Discards a captured graph.  Scratch: 41 B per particle slot of the
 * batch, allocated by the first call with a network.  Errors: QED_ERR_STATE, QED_ERR_ARG (tol not in
 * (0, 1), or the batch's flags hold QED_F_REJECT), QED_ERR_NOMEM. */
qed_status qed_batch_set_mlp(qed_batch_t b, qed_mlp_t m, double tol);
/* For tests of the sampler on the event path: the last step's gathered inputs and samples, the first
 * n_max events (host arrays of n_max doubles each for chi, r, s_beta, n_max x 4 floats for out4, n_max
 * bytes for is_lepton; any may be NULL); *n_out = the number of events of that step; pair events carry
 * placeholder inputs (chi 1, r 1/2, s_beta 0) and is_lepton 0; *n_fallback_total = the samples (pair
 * placeholders included) that took the tables since the network was last set.  Synchronous. */
qed_status qed_batch_mlp_last(qed_batch_t b, int64_t n_max, double *chi, double *r, double *s_beta, float *out4,
                              uint8_t *is_lepton, int64_t *n_out, unsigned long long *n_fallback_total);

/* *begin = *count for each of the n buffers (device-side copy; graph-capturable).  Call it at the start
 * of a time step that runs several step calls, so each call processes only the particles alive when the
 * step began (Sec. 4.3: an event's daughters join the simulation from the next step).  Buffers whose
 * begin is NULL are skipped. */
qed_status qed_snapshot_counts(qed_particles *const *buffers, int32_t n, void *stream);

/* Copy the device counters to host and synchronize `stream` (the only blocking call of a step loop). */
qed_status qed_counters_read(const qed_counters *counters_dev, qed_counters *host_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QED_H */
