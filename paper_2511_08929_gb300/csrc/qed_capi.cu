// qed_capi.cu -- the C ABI of include/qed.h: argument checks, dispatch by buffer layout, and the small
// bookkeeping kernels (birth optical depths, count snapshots and clamps, photon compaction).
#include <atomic>
#include <cstring>

#include "qed_device.cuh"
#include "qed_internal.h"
#include "qed_steps.h"

using namespace qed;

extern "C" int32_t qed_abi_version(void) { return QED_ABI_VERSION; }

extern "C" const char* qed_status_string(int32_t s) {
    switch (s) {
        case QED_OK: return "ok";
        case QED_ERR_ARG: return "invalid argument";
        case QED_ERR_CUDA: return "CUDA runtime error";
        case QED_ERR_CAPACITY: return "particle buffer capacity exhausted";
        case QED_ERR_RANGE: return "chi above table range";
        case QED_ERR_NAN: return "non-finite particle state";
        case QED_ERR_TIMEOUT: return "bounded device wait gave up";
        case QED_ERR_STATE: return "invalid handle";
        case QED_ERR_NOMEM: return "device allocation failed";
        case QED_ERR_TOO_LARGE: return "size above the fixed limit of the call";
        default: return "unknown status";
    }
}

namespace qed {

__global__ void init_tau_kernel(PartDev P, int layout, bool photon, uint64_t seed, int64_t begin) {
    const int64_t n = min(*P.count, P.capacity);
    for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double tau = birth_tau(P.id[i], seed);
        if (layout == QED_FP64) {
            P.tau[i] = tau;
        } else {
            const long long b = __double_as_longlong(tau);
            float4* plane = photon ? P.q1 : P.q2;  // FP32 photons keep tau in q1, leptons in q2
            float4 q = plane[i];
            q.z = __int_as_float((int)(unsigned)(b & 0xffffffffll));
            q.w = __int_as_float((int)(unsigned)((unsigned long long)b >> 32));
            plane[i] = q;
        }
    }
}

struct CountPairs {
    int64_t* count[8];
    int64_t* begin[8];
    int n;
};

__global__ void snapshot_kernel(CountPairs c) {
    const int i = threadIdx.x;
    if (i < c.n) *c.begin[i] = *c.count[i];
}

// the daughter-slot reservation of one step call (AppendState in the caller's counters): opened before
// the step kernel from the daughter buffers' counts, closed after it by advancing the counts
__global__ void append_open_kernel(qed_counters* ctr, const int64_t* c0, int64_t cap0, const int64_t* c1, int64_t cap1) {
    if (threadIdx.x == 0) append_open(append_state(ctr), c0, cap0, c1, cap1);
}

__global__ void append_close_kernel(qed_counters* ctr, int64_t* c0, int64_t* c1) {
    if (threadIdx.x == 0) append_close(append_state(ctr), c0, c1);
}

// ---- compaction (Sec. 4.3: converted photons leave the simulation) ----
struct CompactWs {
    int64_t* holes;  // dead indices below n - D
    int64_t* live;   // live indices in the tail [n - D, n)
    uint8_t* mark;   // tail marks (kept zero between calls)
    int64_t* hdr;    // [0] n, [1] D, [2] holes found, [3] live found
};

inline size_t round16(size_t b) { return (b + 15) & ~size_t(15); }

inline CompactWs carve(void* ws, int64_t cap) {
    char* p = (char*)ws;
    CompactWs w;
    w.hdr = (int64_t*)p;
    p += 64;
    w.holes = (int64_t*)p;
    p += round16(sizeof(int64_t) * cap);
    w.live = (int64_t*)p;
    p += round16(sizeof(int64_t) * cap);
    w.mark = (uint8_t*)p;
    return w;
}

__global__ void compact_head_kernel(PartDev G, CompactWs w) {
    if (threadIdx.x == 0) {
        const int64_t n = max((int64_t)0, min(*G.count, G.capacity));
        w.hdr[0] = n;
        w.hdr[1] = max((int64_t)0, min(*G.n_dead, n));
        w.hdr[2] = 0;
        w.hdr[3] = 0;
    }
}

__global__ void compact_classify_kernel(PartDev G, CompactWs w) {
    const int64_t n = w.hdr[0], D = w.hdr[1], lim = n - D;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < D; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = G.dead[k];
        if (d < 0 || d >= n) continue;
        if (d >= lim) w.mark[d - lim] = 1;
        else w.holes[atomicAdd((unsigned long long*)&w.hdr[2], 1ull)] = d;
    }
}

__global__ void compact_tail_kernel(CompactWs w) {
    const int64_t n = w.hdr[0], D = w.hdr[1], lim = n - D;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x) {
        if (w.mark[i]) w.mark[i] = 0;
        else w.live[atomicAdd((unsigned long long*)&w.hdr[3], 1ull)] = lim + i;
    }
}

__global__ void compact_move_kernel(PartDev G, int layout, CompactWs w) {
    const int64_t nh = min(w.hdr[2], w.hdr[3]);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nh; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = w.live[k], dst = w.holes[k];
        if (layout == QED_FP64) {
            G.x[dst] = G.x[src]; G.y[dst] = G.y[src]; G.z[dst] = G.z[src];
            G.px[dst] = G.px[src]; G.py[dst] = G.py[src]; G.pz[dst] = G.pz[src];
            G.sx[dst] = G.sx[src]; G.sy[dst] = G.sy[src]; G.sz[dst] = G.sz[src];
            G.tau[dst] = G.tau[src]; G.w[dst] = G.w[src];
        } else {
            G.q0[dst] = G.q0[src];
            G.q1[dst] = G.q1[src];
            G.q2[dst] = G.q2[src];
        }
        G.id[dst] = G.id[src];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *G.count = w.hdr[0] - w.hdr[1];
        *G.n_dead = 0;
    }
}

}  // namespace qed

static bool valid_step(const qed_step_desc* s) {
    return s && s->dt > 0.0 && std::isfinite(s->dt) && std::isfinite(s->t) && valid_flags(s->flags) &&
           s->photon_store_min >= 0.0 && s->chi_floor >= 0.0;
}

extern "C" qed_status qed_init_tau(qed_particles* p, uint64_t seed, int64_t begin, void* stream) {
    if (check_particles(p, false) != QED_OK || begin < 0) return QED_ERR_ARG;
    init_tau_kernel<<<launch_blocks(p->capacity, 256), 256, 0, (cudaStream_t)stream>>>(part_dev(p), p->layout,
                                                                                       p->charge == QED_PHOTON, seed, begin);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_snapshot_counts(qed_particles* const* bufs, int32_t n, void* stream) {
    if (n < 0 || (n > 0 && !bufs)) return QED_ERR_ARG;
    CountPairs c{};
    for (int32_t i = 0; i < n; ++i) {
        if (!bufs[i] || !bufs[i]->count) return QED_ERR_ARG;
        if (!bufs[i]->begin) continue;
        if (c.n == 8) {
            snapshot_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(c);
            c.n = 0;
        }
        c.count[c.n] = bufs[i]->count;
        c.begin[c.n] = bufs[i]->begin;
        c.n++;
    }
    if (c.n) snapshot_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(c);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_push_step(qed_tables_t t, const qed_field* field, const qed_step_desc* step,
                                    qed_particles* leptons, qed_particles* photons, qed_counters* ctr, void* stream) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    if (!valid_field(field) || !valid_step(step) || !ctr) return QED_ERR_ARG;
    if (check_particles(leptons, false) != QED_OK || (leptons->charge != QED_ELECTRON && leptons->charge != QED_POSITRON))
        return QED_ERR_ARG;
    if (photons) {
        if (check_particles(photons, false) != QED_OK || photons->layout != leptons->layout ||
            photons->charge != QED_PHOTON || photons->count == leptons->count)
            return QED_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (photons) append_open_kernel<<<1, 32, 0, st>>>(ctr, photons->count, photons->capacity, nullptr, 0);
    if (leptons->layout == QED_FP64) launch_lepton64(t, *field, *step, leptons, photons, ctr, st);
    else launch_lepton32(t, *field, *step, leptons, photons, ctr, st);
    if (photons) append_close_kernel<<<1, 32, 0, st>>>(ctr, photons->count, nullptr);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_pair_step(qed_tables_t t, const qed_field* field, const qed_step_desc* step,
                                    qed_particles* photons, qed_particles* electrons, qed_particles* positrons,
                                    qed_counters* ctr, void* stream) {
    if (!valid_tables(t)) return QED_ERR_STATE;
    if (!valid_field(field) || !valid_step(step) || !ctr) return QED_ERR_ARG;
    if (check_particles(photons, true) != QED_OK || photons->charge != QED_PHOTON) return QED_ERR_ARG;
    if ((electrons == nullptr) != (positrons == nullptr)) return QED_ERR_ARG;
    if (electrons) {
        if (check_particles(electrons, false) != QED_OK || check_particles(positrons, false) != QED_OK ||
            electrons->layout != photons->layout || positrons->layout != photons->layout ||
            electrons->charge != QED_ELECTRON || positrons->charge != QED_POSITRON || electrons->count == positrons->count ||
            electrons->count == photons->count || positrons->count == photons->count)
            return QED_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (electrons)
        append_open_kernel<<<1, 32, 0, st>>>(ctr, electrons->count, electrons->capacity, positrons->count,
                                             positrons->capacity);
    if (photons->layout == QED_FP64) launch_photon64(t, *field, *step, photons, electrons, positrons, ctr, st);
    else launch_photon32(t, *field, *step, photons, electrons, positrons, ctr, st);
    if (electrons) append_close_kernel<<<1, 32, 0, st>>>(ctr, electrons->count, positrons->count);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" size_t qed_compact_workspace_bytes(int64_t capacity) {
    if (capacity < 0) return 0;
    return 64 + 2 * round16(sizeof(int64_t) * (size_t)capacity) + round16((size_t)capacity);
}

extern "C" qed_status qed_compact(qed_particles* photons, void* workspace, size_t bytes, void* stream) {
    if (check_particles(photons, true) != QED_OK || !workspace || !aligned16(workspace) ||
        bytes < qed_compact_workspace_bytes(photons->capacity))
        return QED_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const CompactWs w = carve(workspace, photons->capacity);
    const PartDev g = part_dev(photons);
    const int blocks = launch_blocks(photons->capacity, 256);
    compact_head_kernel<<<1, 32, 0, st>>>(g, w);
    compact_classify_kernel<<<blocks, 256, 0, st>>>(g, w);
    compact_tail_kernel<<<blocks, 256, 0, st>>>(w);
    compact_move_kernel<<<blocks, 256, 0, st>>>(g, photons->layout, w);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_counters_read(const qed_counters* dev, qed_counters* host, void* stream) {
    if (!dev || !host) return QED_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(host, dev, sizeof(qed_counters), cudaMemcpyDeviceToHost, st) != cudaSuccess) return QED_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

// ---- photon compaction without any allocation ----
// qed_compact_noalloc runs the four compaction kernels above on a scratch area that is a file-scope
// device array, sized for QED_COMPACT_NOALLOC_MAX_CAPACITY photons and carved like a caller workspace
// of that capacity.  It serves callers that cannot allocate or hand over device memory at the call
// site: host codes whose device memory is handed out entirely by their own pool, and step loops that
// must stay asynchronous (cudaFree, and cudaMalloc under memory pressure, synchronise the device).
namespace qed {

constexpr size_t kNoAllocScratchBytes =
    64 + 2 * ((sizeof(int64_t) * (size_t)QED_COMPACT_NOALLOC_MAX_CAPACITY + 15) & ~size_t(15)) +
    (((size_t)QED_COMPACT_NOALLOC_MAX_CAPACITY + 15) & ~size_t(15));

// Zero-initialised at module load like every static device object.  A call sets tail marks only in
// [0, D) (D = its dead photons) and its tail kernel clears every mark it reads, so each call leaves the
// marks zero for the next one; the header slots are rewritten by compact_head_kernel.  A call therefore
// costs O(D) like qed_compact, not O(capacity).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocDevices = 64;
static std::atomic<void*> g_noalloc_addr[kNoAllocDevices];

// Device address of the scratch on the current device, looked up once per device.
static cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kNoAllocDevices) {
        void* p = g_noalloc_addr[dev].load(std::memory_order_acquire);
        if (p) {
            *out = p;
            return cudaSuccess;
        }
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kNoAllocDevices) g_noalloc_addr[dev].store(p, std::memory_order_release);
    *out = p;
    return cudaSuccess;
}

}  // namespace qed

extern "C" qed_status qed_compact_noalloc(qed_particles* photons, void* stream) {
    if (check_particles(photons, true) != QED_OK) return QED_ERR_ARG;
    if (photons->capacity > QED_COMPACT_NOALLOC_MAX_CAPACITY) return QED_ERR_TOO_LARGE;
    void* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return QED_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const CompactWs w = carve(scratch, QED_COMPACT_NOALLOC_MAX_CAPACITY);
    const PartDev g = part_dev(photons);
    const int blocks = launch_blocks(photons->capacity, 256);
    compact_head_kernel<<<1, 32, 0, st>>>(g, w);
    compact_classify_kernel<<<blocks, 256, 0, st>>>(g, w);
    compact_tail_kernel<<<blocks, 256, 0, st>>>(w);
    compact_move_kernel<<<blocks, 256, 0, st>>>(g, photons->layout, w);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}
