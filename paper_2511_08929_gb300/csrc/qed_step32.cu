// qed_step32.cu -- the FP32 fast path.
//
// Same algorithm as the FP64 path (Sec. 5.1, 5.2, 6), arithmetic split as follows: the Boris and T-BMT
// pushers, chi, the basis, the rate lookups and all event sampling in FP32; the optical depth is
// accumulated in FP64 and the excess |s|^2 - 1 of a spin / Stokes vector that leaves the unit ball is
// computed in FP64.
//
// GB300 layout and schedule:
//  * particles are three float4 planes (48 B per particle, read and written once per step: the stream
//    is HBM-bound); the id (8 B) is read only when the particle has an event;
//  * every warp walks its own tiles of 32 particles; the next kStages tiles of each plane are brought
//    into shared memory by 1-D bulk copies (cp.async.bulk, completion on an mbarrier per stage), so the
//    loads of later tiles are in flight while the warp computes the current one;
//  * the 1-D rate tables and the Bessel table live in shared memory; the 2-D ICDF tables (<= 1 MB in
//    float) are read through L1/L2 at events only;
//  * a particle whose optical depth runs out is left untouched in global memory by the streaming pass
//    and only its index goes to a per-warp queue; once 32 are queued the warp re-reads them (an L2 hit),
//    recomputes the classical part, and runs the event branch (four Philox draws, the ICDF, Bessel
//    functions, the spectra, the collapses, the daughter append) with all 32 lanes busy.
#include "qed_step32.cuh"

namespace qed {

#ifndef QED_MIN_BLOCKS
#define QED_MIN_BLOCKS 3   // resident blocks per SM the register allocation is sized for
#endif

// ------------------------------------------------------------------------------------------------
// the streaming kernel: per-warp tile pipeline + per-warp event queue (PHOTON selects the species)
// ------------------------------------------------------------------------------------------------
template <bool PHOTON>
__global__ void __launch_bounds__(kT32, QED_MIN_BLOCKS) step32_kernel(TabP<float> T, const float* __restrict__ bes_g,
                                                                      FieldP<float> F, StepP S, float q, PartDev P,
                                                                      PartDev D1, PartDev D2, AppendState* A,
                                                                      Tab64 X, FieldP<double> F64p, qed_counters* ctr) {
    const FieldP<double> F64 = F64p;  // the laser in FP64, for the events taken again in FP64
    extern __shared__ __align__(128) unsigned char smem[];
    const Shared32 sh = carve32(smem, T.n_chi);
    load_tables32(sh, bes_g, T);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TileStream ts;
    ts.tile = sh.tiles + warp * kStages;
    ts.bar = sh.bars + warp * kStages;
    ts.q0 = P.q0;
    ts.q1 = P.q1;
    ts.q2 = P.q2;
    ts.n = min(P.begin ? *P.begin : *P.count, P.capacity);
    ts.g0 = (int64_t)blockIdx.x * kWarps32 + warp;
    ts.G = (int64_t)gridDim.x * kWarps32;
    int64_t* wq = sh.queue + warp * kWQ;
    if (lane == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&ts.bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();  // tables and barriers ready
    Ctx C;
    C.T = T;
    C.T.nlc_rate = sh.rates;
    C.T.nbw_rate = sh.rates + 2 * T.n_chi;
    C.bes = sh.bes;
    C.F = F;
    C.S = S;
    C.q = q;
    unsigned long long c[C_N] = {};
    if (lane == 0)
        for (int s = 0; s < kStages; ++s) ts.issue(s);
    int qn = 0;  // queued event indices (warp-uniform)
    int64_t t = 0;
    bool timed_out = false;
    for (; ts.base(t) < ts.n; ++t) {
        const int s = (int)(t % kStages);
        if (!mbar_wait(&ts.bar[s], (uint32_t)((t / kStages) & 1))) {
            timed_out = true;
            break;
        }
        const int64_t j = ts.base(t) + lane;
        const bool valid = j < ts.n;
        float4 a = make_float4(0, 0, 0, 0), b = a, cc = a;
        if (valid) {
            a = ts.tile[s].q0[lane];
            b = ts.tile[s].q1[lane];
            cc = ts.tile[s].q2[lane];
        }
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async();  // this stage's reads happen before the next copy overwrites it
            ts.issue(t + kStages);
        }
        bool event = false;
        if (valid)
            event = PHOTON ? photon_stream_one(C, P, j, a, b, cc, ctr, c) : lepton_stream_one(C, P, j, a, b, cc, ctr, c);
        const unsigned m = __ballot_sync(0xffffffffu, event);
        if (event) wq[qn + __popc(m & ((1u << lane) - 1u))] = j;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
            const int64_t je = wq[qn - 32 + lane];
            if (PHOTON) photon_events(C, X, je, P, D1, D2, A, ctr, c);
            else lepton_events(C, X, F64, je, P, D1, A, ctr, c);
            qn -= 32;
            __syncwarp();
        }
    }
    if (timed_out) {
        if (lane == 0) {
            record_error(ctr, QED_ERR_TIMEOUT, ts.base(t));
            for (int64_t u = t; u < t + kStages && ts.base(u) < ts.n; ++u)  // let the copies in flight land
                mbar_wait(&ts.bar[u % kStages], (uint32_t)((u / kStages) & 1));
        }
        __syncwarp();
    }
    if (qn > 0) {
        const int64_t je = lane < qn ? wq[lane] : -1;
        if (PHOTON) photon_events(C, X, je, P, D1, D2, A, ctr, c);
        else lepton_events(C, X, F64, je, P, D1, A, ctr, c);
    }
    flush_warp(c, ctr);
}

}  // namespace qed

// grid = SMs x resident blocks of the kernel (persistent loop over tiles); cached per kernel
struct Launch32 {
    const void* kern = nullptr;
    size_t smem = 0;
    int blocks = 0;
};

static int blocks32(int64_t capacity, const void* kern, size_t smem) {
    static Launch32 cache[2];
    Launch32* e = nullptr;
    for (auto& c : cache)
        if (c.kern == kern || c.kern == nullptr) {
            e = &c;
            break;
        }
    if (e->kern != kern || e->smem != smem) {
        int dev = 0, sms = 1, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, qed::kT32, smem);
        e->kern = kern;
        e->smem = smem;
        e->blocks = sms * (per_sm < 1 ? 1 : per_sm);
    }
    const int64_t need = (capacity + 31) / 32;  // tiles of 32 particles
    return (int)std::max<int64_t>(1, std::min<int64_t>((need + qed::kWarps32 - 1) / qed::kWarps32, (int64_t)e->blocks));
}

void launch_lepton32(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* L,
                     const qed_particles* G, qed_counters* ctr, cudaStream_t st) {
    using namespace qed;
    const size_t smem = smem32_bytes(t->desc.n_chi);
    PartDev g{};
    if (G) g = part_dev(G);
    const void* k = (const void*)step32_kernel<false>;
    step32_kernel<false><<<blocks32(L->capacity, k, smem), kT32, smem, st>>>(
        tab_params<float>(t), t->bes32, field_params<float>(f), step_params(s, f), (float)L->charge, part_dev(L), g,
        PartDev{}, G ? append_state(ctr) : nullptr, Tab64{tab_params<double>(t), t->bes64}, field_params<double>(f), ctr);
}

void launch_photon32(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* G,
                     const qed_particles* El, const qed_particles* Po, qed_counters* ctr, cudaStream_t st) {
    using namespace qed;
    const size_t smem = smem32_bytes(t->desc.n_chi);
    PartDev e{}, p{};
    if (El && Po) {
        e = part_dev(El);
        p = part_dev(Po);
    }
    const void* k = (const void*)step32_kernel<true>;
    step32_kernel<true><<<blocks32(G->capacity, k, smem), kT32, smem, st>>>(
        tab_params<float>(t), t->bes32, field_params<float>(f), step_params(s, f), 0.0f, part_dev(G), e, p,
        (El && Po) ? append_state(ctr) : nullptr, Tab64{tab_params<double>(t), t->bes64}, field_params<double>(f), ctr);
}
