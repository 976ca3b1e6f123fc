// qed_batch.cu -- batched collisions: every instance and species of a batch in one persistent launch per
// time step, the step index and time on the device (so a CUDA graph of whole steps replays unchanged),
// and an autotuner for the launch shape.
//
// One time step of the batch is seven launches on one stream:
//   plan      alive counts at step start (counts clamped to capacity), the tile list over all segments
//             (segment = one species of one instance, species-major), each segment's step context,
//             particle-step accounting;
//   step      the persistent kernel: every warp takes runs of consecutive tiles from a work counter
//             (guided: long runs first, short ones at the end, at most `chunk` tiles) and streams them
//             through shared memory with per-lane asynchronous copies, running the per-particle
//             arithmetic of the single-buffer FP32 kernels;
//             a particle whose optical depth runs out is left untouched and listed (segment, index) in
//             the step's event list, 32 entries per atomic add;
//   events    the event branch for every listed particle, 32 per warp with a context per lane (out of
//             the persistent kernel, whose registers then hold only the streaming pass: no calls, no
//             spills);
//   compact   head / classify / tail / move of every instance's photons (converted photons leave,
//             Sec. 4.3), the last one also advancing the device step counter.
// Daughters appended during a step sit beyond the counts taken by `plan`, so they are first stepped in
// the next step (the begin snapshot of the single-buffer path).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

// the event kernel runs the event passes inline (measured 21 % faster than out-of-line calls at the
// same occupancy: the calls' register saves and frames went through local memory)
#define QED_EVENT_PASS __forceinline__
#include "qed_step32.cuh"

namespace qed {

constexpr int kSpecies = 3;  // electrons, positrons, photons

struct InstDev {
    FieldP<float> F;
    FieldP<double> F64;  // the same laser in FP64 (events taken again in FP64)
    double phase;
    uint64_t seed;
    PartDev sp[kSpecies];
    int64_t* holes;  // photon compaction scratch of this instance
    int64_t* live;
    uint8_t* mark;
    int64_t* hdr;  // [0] n, [1] D, [2] holes found, [3] live found
    AppendState* app;  // daughter reservations of the step: [0] photons (lepton events), [1] pairs
};

struct SegDev {
    const float4 *q0, *q1, *q2;
    int64_t n;  // particles processed this step
};

struct ClockDev {
    uint64_t step, step0;
    double t0, dt;
    unsigned long long psteps;
    unsigned long long species_steps[kSpecies];
    long long alive[kSpecies];
    int next_tile;  // the persistent kernel's work counter (tiles handed out), reset by the plan kernel
    unsigned long long n_events;  // entries in the step's event list, reset by the plan kernel
};

struct BatchP {
    uint32_t flags;
    float dt_f;
    double store_min, chi_floor;
};

// The step context of one segment (one species of one instance), written by the plan kernel every
// step for the event kernel: its lanes take events of several segments at once.
struct SegCtx {
    Ctx C;       // tables (global memory), field, step parameters and charge
    int ii, sp;  // instance and species
};

// ------------------------------------------------------------------------------------------------
// plan: one block of kPlanThreads threads, each owning up to 3 consecutive segments
// ------------------------------------------------------------------------------------------------
constexpr int kPlanThreads = 1024;

__global__ void __launch_bounds__(kPlanThreads)
    batch_plan_kernel(const InstDev* __restrict__ inst, int n_inst, SegDev* seg, int64_t* tile0, ClockDev* clk,
                      SegCtx* ctx, TabP<float> T, const float* bes, BatchP P) {
    __shared__ long long wsum[32];
    __shared__ unsigned long long tot[kSpecies];
    const int n_seg = kSpecies * n_inst;
    const int per = (n_seg + kPlanThreads - 1) / kPlanThreads;  // <= 3
    const int s0 = threadIdx.x * per;
    if (threadIdx.x < kSpecies) tot[threadIdx.x] = 0;
    __syncthreads();
    long long loc[3] = {0, 0, 0}, mine = 0;
    for (int k = 0; k < per; ++k) {
        const int s = s0 + k;
        if (s >= n_seg) break;
        const int sp = s / n_inst, i = s - sp * n_inst;
        const PartDev& Pd = inst[i].sp[sp];
        const int64_t c = *Pd.count;
        const int64_t n = c < 0 ? 0 : (c > Pd.capacity ? Pd.capacity : c);
        if (c != n) *Pd.count = n;  // reservations that did not fit
        seg[s] = SegDev{Pd.q0, Pd.q1, Pd.q2, n};
        loc[k] = (n + 31) / 32;
        mine += loc[k];
        atomicAdd(&tot[sp], (unsigned long long)n);
    }
    // block-wide exclusive scan of the per-thread tile counts
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long v = wsum[lane], x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        wsum[lane] = x - v;  // exclusive prefix of the warp totals
        if (lane == 31) tile0[n_seg] = x;
    }
    __syncthreads();
    long long ex = wsum[wid] + incl - mine;
    const uint64_t step = clk->step;
    // time of this step: a product then a sum, each rounded (no contraction)
    const double t_now = __dadd_rn(clk->t0, __dmul_rn((double)(step - clk->step0), clk->dt));
    for (int k = 0; k < per; ++k) {
        const int s = s0 + k;
        if (s >= n_seg) break;
        tile0[s] = ex;
        ex += loc[k];
        const int sp = s / n_inst, i = s - sp * n_inst;
        const InstDev& I = inst[i];
        SegCtx& X = ctx[s];
        X.ii = i;
        X.sp = sp;
        X.C.T = T;
        X.C.bes = bes;
        X.C.F = I.F;
        X.C.q = sp == 0 ? -1.0f : (sp == 1 ? 1.0f : 0.0f);
        StepP& S = X.C.S;
        S.dt = clk->dt;
        S.ph_hi = __dadd_rn(t_now, I.phase);
        S.ph_hi_f = (float)S.ph_hi;
        S.ph_lo_f = (float)(S.ph_hi - (double)S.ph_hi_f);
        S.dt_f = P.dt_f;
        S.flags = P.flags;
        S.step = step;
        S.seed = I.seed;
        S.store_min = P.store_min;
        S.chi_floor = P.chi_floor;
        S.store_min_f = (float)P.store_min;
        S.chi_floor_f = (float)P.chi_floor;
    }
    // open every instance's daughter reservations from the counts at step start (clamped above)
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        const InstDev& I = inst[i];
        append_open(&I.app[0], I.sp[2].count, I.sp[2].capacity, nullptr, 0);
        append_open(&I.app[1], I.sp[0].count, I.sp[0].capacity, I.sp[1].count, I.sp[1].capacity);
    }
    if (threadIdx.x == 0) {
        clk->next_tile = 0;
        clk->n_events = 0;
        clk->psteps += tot[0] + tot[1] + tot[2];
        for (int k = 0; k < kSpecies; ++k) {
            clk->species_steps[k] += tot[k];
            clk->alive[k] = (long long)tot[k];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// the persistent step kernel
// ------------------------------------------------------------------------------------------------

// Guided self-scheduling of the tile list: a warp takes [start, start + size) from the work counter
// with one atomic add, size = (tiles not yet handed out by its last take) / (2 x warps), clamped to
// [min(kMinChunk, chunk), chunk].  Early takes are long runs of consecutive tiles (few segment changes), the last
// ones short, so the warps finish together whatever the cost of their tiles.  Takes return increasing
// starts, so every warp walks the tile list forward.  The copy walk (lane 0) takes the chunks one ahead
// and passes their bounds to the compute walk through a per-warp ring in shared memory.
constexpr int kMinChunk = 2;
constexpr int kChunkRing = 8;  // > STAGES + 1: the chunks between the compute and the copy walks

__device__ __forceinline__ int guided_size(int total, int from, int warps2, int chunk) {
    const int left = total - from;
    const int g = left > 0 ? left / warps2 : 0;
    const int lo = chunk < kMinChunk ? chunk : kMinChunk;
    return g < lo ? lo : (g > chunk ? chunk : g);
}

// per-thread asynchronous 16-byte copies global -> shared (cp.async, L2 only), committed and awaited in
// groups: every lane copies its own particle of a tile and later reads only what it copied itself
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// all lanes: start the copies of tile t into stage st (one commit group), moving the copy cursor cs
// (segment of the last issued tile; tiles only increase) forward
__device__ __forceinline__ void batch_issue(Tile* tile, const int* tile0, const SegDev* __restrict__ seg, int t, int st,
                                            int& cs) {
    while (tile0[cs + 1] <= t) ++cs;
    const SegDev g = seg[cs];
    const int j = (t - tile0[cs]) * 32 + (threadIdx.x & 31);
    if (j < g.n) {
        const int l = threadIdx.x & 31;
        cp_async16(&tile[st].q0[l], g.q0 + j);
        cp_async16(&tile[st].q1[l], g.q1 + j);
        cp_async16(&tile[st].q2[l], g.q2 + j);
    }
    cp_async_commit();
}

// per-warp state of the current segment, in shared memory (written by lane 0 at a segment change)
struct WarpSeg {
    Ctx C;      // tables, field, step parameters and charge of the segment's instance and species
    PartDev L;  // the segment's buffer (planes, ids, count) for the streaming pass
    int t0, t1, n;  // its tile range and particle count
};

// shared memory of the batched kernel: the 1-D rate tables (the Bessel table, read only by the event
// kernel, stays in global memory behind L1), the tile list, the per-warp segment state, the tiles, the
// event queues and the chunk rings
__host__ __device__ inline size_t batch_smem_bytes(int warps, int stages, int n_chi, int n_seg) {
    size_t off = align128((size_t)4 * n_chi * 4);
    off += align128((size_t)(n_seg + 1) * 4);
    off += align128((size_t)warps * sizeof(WarpSeg));
    off += (size_t)warps * stages * sizeof(Tile);
    off += (size_t)warps * kWQ * 8;
    off += (size_t)warps * kChunkRing * 8;
    return off;
}

// FIX: the step flags fixed at compile time (0: read from the context)
template <int WARPS, int STAGES, int MINB, uint32_t FIX>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    batch_step_kernel(TabP<float> T, float* bes_g, const InstDev* __restrict__ inst,
                      const SegDev* __restrict__ seg, const int64_t* __restrict__ tile0_g, int n_inst,
                      const ClockDev* __restrict__ clk, BatchP P, int chunk, int* work, long long* ev,
                      unsigned long long* n_ev, qed_counters* ctr) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int n_seg = kSpecies * n_inst;
    Shared32 sh;
    sh.bes = bes_g;
    sh.rates = (float*)smem;
    size_t off = align128((size_t)4 * T.n_chi * 4);
    int* s_tile0 = (int*)(smem + off);
    off += align128((size_t)(n_seg + 1) * 4);
    WarpSeg* s_ws = (WarpSeg*)(smem + off);
    off += align128((size_t)WARPS * sizeof(WarpSeg));
    sh.tiles = (Tile*)(smem + off);
    off += (size_t)WARPS * STAGES * sizeof(Tile);
    sh.bars = nullptr;
    sh.queue = (int64_t*)(smem + off);
    off += (size_t)WARPS * kWQ * 8;
    int2* s_chunks = (int2*)(smem + off);

    for (int i = threadIdx.x; i < 2 * T.n_chi; i += blockDim.x) {
        sh.rates[i] = T.nlc_rate[i];
        sh.rates[2 * T.n_chi + i] = T.nbw_rate[i];
    }
    for (int i = threadIdx.x; i <= n_seg; i += blockDim.x) s_tile0[i] = (int)tile0_g[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Tile* tile = sh.tiles + warp * STAGES;
    int64_t* wq = sh.queue + warp * kWQ;
    WarpSeg& WS = s_ws[warp];
    Ctx& C = WS.C;
    if (lane == 0) WS.t1 = 0;
    __syncthreads();  // tables and tile list ready
    const int total = s_tile0[n_seg];
    // the tables as the streaming pass reads them: the kernel's parameters, with the rate rows in shared
    // memory (the segment contexts in shared memory keep a copy for the event branch)
    TabP<float> Tl = T;
    Tl.nlc_rate = sh.rates;
    Tl.nbw_rate = sh.rates + 2 * T.n_chi;
    const int W2 = 2 * gridDim.x * WARPS;
    unsigned long long c[C_N] = {};
    int2* ring = s_chunks + warp * kChunkRing;
    // the copy walk (warp-uniform): tile pt of a chunk ending at pe, the chunks put in the ring (pk), the
    // prefetched take (ns, nsz; lane 0 adds, the warp shares the result)
    int pt, pe, pk = 0, ns = total, nsz = 0;
    int cs = 0;
    {
        const int sz = guided_size(total, 0, W2, chunk);
        const int s0 = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(work, sz) : 0, 0);
        pt = min(s0, total);
        pe = min(s0 + sz, total);
        if (lane == 0) ring[pk & (kChunkRing - 1)] = make_int2(pt, pe);
        ++pk;
        if (pt < pe) {
            nsz = guided_size(total, s0, W2, chunk);
            ns = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(work, nsz) : 0, 0);
        }
        for (int s = 0; s < STAGES; ++s) {
            if (pt < pe) {
                batch_issue(tile, s_tile0, seg, pt, s, cs);
                if (++pt == pe) {  // the chunk is issued: take the prefetched one
                    pt = min(ns, total);
                    pe = min(ns + nsz, total);
                    if (lane == 0) ring[pk & (kChunkRing - 1)] = make_int2(pt, pe);
                    ++pk;
                    if (pt < pe) {
                        const int from = ns;
                        nsz = guided_size(total, from, W2, chunk);
                        ns = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(work, nsz) : 0, 0);
                    }
                }
            } else {
                cp_async_commit();  // an empty group keeps one group per stage
            }
        }
    }
    __syncwarp();
    int2 ch = ring[0];
    int t = ch.x, te = ch.y, rk = 1;  // the compute walk: tile t of a chunk ending at te; ring entries read
    int qn = 0;    // queued event entries, segment << 32 | index (warp-uniform), flushed 32 at a time
    int cur = -1;  // current segment
    int sp = 0, ii = 0;
    int st = 0;  // stage of the current tile
    while (t < te) {
        cp_async_wait<STAGES - 1>();  // this lane's copies of the current tile have landed
        if (t >= WS.t1) {  // the tile lies in a later segment
            do ++cur;
            while (s_tile0[cur + 1] <= t);
            sp = cur / n_inst;
            ii = cur - sp * n_inst;
            __syncwarp();
            if (lane == 0) {
                const InstDev& I = inst[ii];
                const uint64_t step = clk->step;
                // time of this step: a product then a sum, each rounded (no contraction)
                const double t_now = __dadd_rn(clk->t0, __dmul_rn((double)(step - clk->step0), clk->dt));
                WS.t0 = s_tile0[cur];
                WS.t1 = s_tile0[cur + 1];
                WS.n = (int)seg[cur].n;
                WS.L = I.sp[sp];
                C.T = T;
                C.T.nlc_rate = sh.rates;
                C.T.nbw_rate = sh.rates + 2 * T.n_chi;
                C.bes = sh.bes;
                C.F = I.F;
                C.q = sp == 0 ? -1.0f : (sp == 1 ? 1.0f : 0.0f);
                StepP S;
                S.dt = clk->dt;
                S.ph_hi = __dadd_rn(t_now, I.phase);
                S.ph_hi_f = (float)S.ph_hi;
                S.ph_lo_f = (float)(S.ph_hi - (double)S.ph_hi_f);
                S.dt_f = P.dt_f;
                S.flags = P.flags;
                S.step = step;
                S.seed = I.seed;
                S.store_min = P.store_min;
                S.chi_floor = P.chi_floor;
                S.store_min_f = (float)P.store_min;
                S.chi_floor_f = (float)P.chi_floor;
                C.S = S;
            }
            __syncwarp();
        }
        const int j = (t - WS.t0) * 32 + lane;
        const bool valid = j < WS.n;
        float4 a = make_float4(0, 0, 0, 0), b = a, cc = a;
        if (valid) {
            a = tile[st].q0[lane];
            b = tile[st].q1[lane];
            cc = tile[st].q2[lane];
        }
        if (pt < pe) {  // the copies of the tile STAGES ahead, into the stage just read
            batch_issue(tile, s_tile0, seg, pt, st, cs);
            if (++pt == pe) {  // the chunk is issued: take the prefetched one
                pt = min(ns, total);
                pe = min(ns + nsz, total);
                if (lane == 0) ring[pk & (kChunkRing - 1)] = make_int2(pt, pe);
                ++pk;
                if (pt < pe) {
                    const int from = ns;
                    nsz = guided_size(total, from, W2, chunk);
                    ns = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(work, nsz) : 0, 0);
                }
            }
        } else {
            cp_async_commit();
        }
        if (++st == STAGES) st = 0;
        bool event = false;
        if (valid)
            event = sp == 2 ? photon_stream_one<FIX>(C, WS.L, j, a, b, cc, ctr, c, &Tl)
                            : lepton_stream_one<FIX>(C, WS.L, j, a, b, cc, ctr, c, &Tl);
        const unsigned m = __ballot_sync(0xffffffffu, event);
        if (event) wq[qn + __popc(m & ((1u << lane) - 1u))] = ((long long)cur << 32) | (long long)j;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {  // 32 entries to the step's event list with one atomic add
            const unsigned long long base = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(n_ev, 32ull) : 0ull, 0);
            ev[base + lane] = wq[qn - 32 + lane];
            qn -= 32;
            __syncwarp();
        }
        if (++t == te) {  // the chunk is done: the next one (its entry was written when its copies began)
            ch = ring[rk++ & (kChunkRing - 1)];
            t = ch.x;
            te = ch.y;
        }
    }
    cp_async_wait<0>();  // no copy outlives the kernel (the trailing groups are empty)
    if (qn > 0) {
        const unsigned long long base =
            __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(n_ev, (unsigned long long)qn) : 0ull, 0);
        if (lane < qn) ev[base + lane] = wq[lane];
    }
    flush_warp(c, ctr);
}

// ------------------------------------------------------------------------------------------------
// the event pass of the step: every event the persistent kernel listed (a particle whose optical depth
// ran out, left untouched by it), 32 per warp, each lane with the context of its own segment
// ------------------------------------------------------------------------------------------------
constexpr int kEventThreads = 256;

// (two blocks per SM: the register cap keeps 16 warps per SM to hide the global-memory latency of the
// event branch)
__global__ void __launch_bounds__(kEventThreads, 2) batch_event_kernel(const InstDev* __restrict__ inst,
                                                                   const SegCtx* __restrict__ ctx,
                                                                   const long long* __restrict__ ev,
                                                                   const ClockDev* __restrict__ clk, Tab64 X64,
                                                                   qed_counters* ctr,
                                                                   const float* __restrict__ lnup = nullptr) {
    __shared__ ExactQ eq[kEventThreads / 32];  // per warp: the events taken again in FP64
    const unsigned long long n = clk->n_events;
    unsigned long long c[C_N] = {};
    const int lane = threadIdx.x & 31;
    ExactQ& q = eq[threadIdx.x >> 5];
    if (lane == 0) q.n = 0;
    __syncwarp();
    // lanes take queued entries [from, from + cnt), each with the context of its own segment
    auto drain = [&](int from, int cnt) {
        if (lane < cnt) {
            const int key = q.key[from + lane];
            const SegCtx& X = ctx[key & 0x3FFFFFFF];
            const InstDev& I = inst[X.ii];
            lepton_exact_one(X.C, X64, I.F64, I.sp[X.sp], I.sp[2], q.j[from + lane], q.slot[from + lane],
                             (key >> 30) & 1, lnup != nullptr, q.lnu[from + lane]);
        }
        __syncwarp();
    };
    const unsigned long long warps = (unsigned long long)gridDim.x * (kEventThreads / 32);
    for (unsigned long long k = ((unsigned long long)blockIdx.x * (kEventThreads / 32) + (threadIdx.x >> 5)) * 32; k < n;
         k += warps * 32) {
        const long long e = k + lane < n ? ev[k + lane] : -1;
        const int seg0 = __shfl_sync(0xffffffffu, (int)(e >> 32), 0);  // lane 0 always holds an entry
        const int s = e >= 0 ? (int)(e >> 32) : seg0;
        const int64_t j = e >= 0 ? (int64_t)(uint32_t)e : -1;
        const SegCtx& X = ctx[s];
        const InstDev& I = inst[X.ii];
        const bool ph = X.sp == 2;
        const float lnu = lnup != nullptr && e >= 0 ? lnup[4 * (k + lane)] : 0.0f;  // the learned sampler's ln u'
        // both passes are warp-collective; a lane takes part in the one of its species with its particle
        if (__ballot_sync(0xffffffffu, j >= 0 && !ph))
            lepton_events(X.C, X64, I.F64, ph ? -1 : j, I.sp[ph ? 0 : X.sp], I.sp[2], &I.app[0], ctr, c, &q, s,
                          lnup != nullptr, lnu);
        if (__ballot_sync(0xffffffffu, j >= 0 && ph))
            photon_events(X.C, X64, ph ? j : -1, I.sp[2], I.sp[0], I.sp[1], &I.app[1], ctr, c);
        const int qn = q.n;
        if (qn >= 32) {  // 32 queued events in FP64 with every lane busy
            drain(qn - 32, 32);
            if (lane == 0) q.n = qn - 32;
            __syncwarp();
        }
    }
    drain(0, q.n);
    flush_warp(c, ctr);
}

// ------------------------------------------------------------------------------------------------
// the learned sampler's inputs for every listed event (Sec. 5.1): a lepton's (chi, r2, s.beta) as its
// event will see them (the streaming pass's classical step with accurate fields; r2 the uniform of its
// energy-fraction draw, which the ICDF row would take); a pair event gets placeholders (chi 1, r 1/2,
// s 0) and lep 0, so that list position k is sample k
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) batch_mlp_prep_kernel(const InstDev* __restrict__ inst,
                                                             const SegCtx* __restrict__ ctx,
                                                             const long long* __restrict__ ev,
                                                             const ClockDev* __restrict__ clk, double* chi, double* r,
                                                             double* sb, uint8_t* lep) {
    const unsigned long long n = clk->n_events;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const long long e = ev[k];
        const SegCtx& X = ctx[(int)(e >> 32)];
        if (X.sp == 2) {
            chi[k] = 1.0;
            r[k] = 0.5;
            sb[k] = 0.0;
            lep[k] = 0;
            continue;
        }
        const int64_t j = (int64_t)(uint32_t)e;
        const PartDev& L = inst[X.ii].sp[X.sp];
        const float4 a = __ldcg(L.q0 + j), b = __ldcg(L.q1 + j), cc = __ldcg(L.q2 + j);
        LState st;
        lepton_classical<0, true>(X.C, a, b, cc, st, nullptr);
        const uint4 w1 = draw(L.id[j], X.C.S.seed, X.C.S.step, kSlotLambdaSpin);
        chi[k] = (double)st.chi;
        r[k] = uniform52(w1.x, w1.y);
        sb[k] = (double)st.sb;
        lep[k] = 1;
    }
}

// ------------------------------------------------------------------------------------------------
// photon compaction of every instance (grid.y = instance); the same hole filling as qed_compact
// ------------------------------------------------------------------------------------------------
constexpr int kCompactBlocks = 8;  // blocks per instance (grid-stride over the dead list)

__global__ void batch_compact_head(const InstDev* __restrict__ inst, int n_inst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const InstDev& I = inst[i];
    const PartDev& G = I.sp[2];
    // close the step's daughter reservations: the counts after this step's appends
    append_close(&I.app[0], G.count, nullptr);
    append_close(&I.app[1], I.sp[0].count, I.sp[1].count);
    const int64_t n = max((int64_t)0, min(*G.count, G.capacity));
    I.hdr[0] = n;
    I.hdr[1] = max((int64_t)0, min(*G.n_dead, n));
    I.hdr[2] = 0;
    I.hdr[3] = 0;
}

__global__ void batch_compact_classify(const InstDev* __restrict__ inst) {
    const InstDev& I = inst[blockIdx.y];
    const int64_t n = I.hdr[0], D = I.hdr[1], lim = n - D;
    const int64_t* dead = I.sp[2].dead;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < D; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = dead[k];
        if (d < 0 || d >= n) continue;
        if (d >= lim) I.mark[d - lim] = 1;
        else I.holes[atomicAdd((unsigned long long*)&I.hdr[2], 1ull)] = d;
    }
}

__global__ void batch_compact_tail(const InstDev* __restrict__ inst) {
    const InstDev& I = inst[blockIdx.y];
    const int64_t n = I.hdr[0], D = I.hdr[1], lim = n - D;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < D; k += (int64_t)gridDim.x * blockDim.x) {
        if (I.mark[k]) I.mark[k] = 0;
        else I.live[atomicAdd((unsigned long long*)&I.hdr[3], 1ull)] = lim + k;
    }
}

__global__ void batch_compact_move(const InstDev* __restrict__ inst, ClockDev* clk) {
    const InstDev& I = inst[blockIdx.y];
    const PartDev& G = I.sp[2];
    const int64_t nh = min(I.hdr[2], I.hdr[3]);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nh; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = I.live[k], dst = I.holes[k];
        G.q0[dst] = G.q0[src];
        G.q1[dst] = G.q1[src];
        G.q2[dst] = G.q2[src];
        G.id[dst] = G.id[src];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *G.count = I.hdr[0] - I.hdr[1];
        *G.n_dead = 0;
        if (blockIdx.y == 0) clk->step += 1;  // the step is complete: advance the device clock
    }
}

}  // namespace qed

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
using namespace qed;

constexpr uint32_t kBatchMagic = 0x51454442u;  // "QEDB"

struct qed_batch_s;
typedef void (*batch_launch_fn)(const qed_batch_s* b, int grid, cudaStream_t st);

struct BatchVariant {
    const void* kern;
    int warps, stages;
    batch_launch_fn launch;
};

struct qed_batch_s {
    uint32_t magic;
    int device, sms;
    const qed_tables_s* tables;
    int n_inst;
    bool plane_waves;  // every instance a single plane wave (LP or CP): the fixed-flag kernels may run it
    qed_batch_desc desc;
    qed_counters* ctr;
    InstDev* d_inst;
    SegDev* d_seg;
    SegCtx* d_ctx;     // per-segment step contexts (plan kernel -> event kernel)
    long long* d_ev;   // the step's event list: segment << 32 | particle index, one slot per particle
    int ev_grid;       // event kernel grid
    int64_t* d_tile0;
    ClockDev* d_clk;
    int64_t* d_hdr;
    AppendState* d_app;  // two daughter reservations per instance
    unsigned char* d_ws;
    int64_t capacity_total;
    qed_batch_tuning tuning;
    int grid;  // persistent grid of the current tuning
    cudaStream_t cap_stream;
    cudaGraphExec_t exec;
    int exec_steps;
    std::vector<cudaEvent_t> kev;  // caller's event pairs around the persistent kernel (may be empty)
    long long direct_steps;        // directly launched steps (event pair index of the next one)
    // the learned sampler on the event path (mlp NULL: the tables): per listed event its inputs, the
    // sampler's outputs and whether it is a lepton's; the fallback count since the network was set
    qed_mlp_t mlp;
    double mlp_tol;
    int mlp_grid;
    double *d_mchi, *d_mr, *d_ms;
    float* d_mout;
    uint8_t* d_mlep;
    unsigned long long* d_mfb;
};

template <int WARPS, int STAGES, int MINB, uint32_t FIX>
static void launch_variant(const qed_batch_s* b, int grid, cudaStream_t st) {
    const qed_tables_s* t = b->tables;
    const size_t smem = batch_smem_bytes(WARPS, STAGES, t->desc.n_chi, kSpecies * b->n_inst);
    BatchP P;
    P.flags = b->desc.flags;
    P.dt_f = (float)b->desc.dt;
    P.store_min = b->desc.photon_store_min;
    P.chi_floor = b->desc.chi_floor;
    batch_step_kernel<WARPS, STAGES, MINB, FIX><<<grid, WARPS * 32, smem, st>>>(
        tab_params<float>(t), t->bes32, b->d_inst, b->d_seg, b->d_tile0, b->n_inst, b->d_clk, P, b->tuning.chunk,
        &b->d_clk->next_tile, b->d_ev, &b->d_clk->n_events, b->ctr);
}

#define QED_VARIANTS(FIX)                                                                \
    {{(const void*)batch_step_kernel<8, 3, 3, FIX>, 8, 3, launch_variant<8, 3, 3, FIX>},      \
     {(const void*)batch_step_kernel<8, 3, 2, FIX>, 8, 3, launch_variant<8, 3, 2, FIX>},      \
     {(const void*)batch_step_kernel<8, 2, 4, FIX>, 8, 2, launch_variant<8, 2, 4, FIX>},      \
     {(const void*)batch_step_kernel<16, 2, 1, FIX>, 16, 2, launch_variant<16, 2, 1, FIX>},   \
     {(const void*)batch_step_kernel<16, 2, 2, FIX>, 16, 2, launch_variant<16, 2, 2, FIX>}}

// [0]: flags read at run time; [1]: built for QED_F_FULL (every flag test of the streaming pass folded)
static const BatchVariant kVariants[2][QED_BATCH_VARIANTS] = {QED_VARIANTS(0u), QED_VARIANTS(QED_F_FULL)};

static const BatchVariant& variant_of(const qed_batch_s* b, int v) {
    return kVariants[b->desc.flags == QED_F_FULL && b->plane_waves ? 1 : 0][v];
}

static size_t variant_smem(const qed_batch_s* b, int v) {
    return batch_smem_bytes(variant_of(b, v).warps, variant_of(b, v).stages, b->tables->desc.n_chi, kSpecies * b->n_inst);
}

// resident blocks per SM of variant v for this batch (0 if it does not fit)
static int variant_occupancy(const qed_batch_s* b, int v) {
    int per_sm = 0;
    const size_t smem = variant_smem(b, v);
    const BatchVariant& k = variant_of(b, v);
    if (cudaFuncSetAttribute(k.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.kern, k.warps * 32, smem) != cudaSuccess) return 0;
    return per_sm;
}

static bool valid_batch(const qed_batch_s* b) { return b != nullptr && b->magic == kBatchMagic; }

// one time step of the batch on `st`; e0 / e1 (may be null) are recorded around the persistent kernel
// (as event-record nodes of the graph when `st` is capturing)
static void launch_batch_step(const qed_batch_s* b, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                              bool capturing = false) {
    const unsigned rec = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    BatchP P;
    P.flags = b->desc.flags;
    P.dt_f = (float)b->desc.dt;
    P.store_min = b->desc.photon_store_min;
    P.chi_floor = b->desc.chi_floor;
    batch_plan_kernel<<<1, kPlanThreads, 0, st>>>(b->d_inst, b->n_inst, b->d_seg, b->d_tile0, b->d_clk, b->d_ctx,
                                                  tab_params<float>(b->tables), b->tables->bes32, P);
    if (e0) cudaEventRecordWithFlags(e0, st, rec);
    variant_of(b, b->tuning.variant).launch(b, b->grid, st);
    if (b->mlp) {  // the learned sampler draws every listed emission's energy fraction
        batch_mlp_prep_kernel<<<b->sms * 8, 256, 0, st>>>(b->d_inst, b->d_ctx, b->d_ev, b->d_clk, b->d_mchi, b->d_mr,
                                                          b->d_ms, b->d_mlep);
        mlp_sample_listed(b->mlp, b->tables, b->d_mchi, b->d_mr, b->d_ms, b->capacity_total, &b->d_clk->n_events,
                          b->mlp_tol, b->d_mout, b->d_mfb, b->mlp_grid, st);
    }
    batch_event_kernel<<<b->ev_grid, kEventThreads, 0, st>>>(b->d_inst, b->d_ctx, b->d_ev, b->d_clk,
                                                             Tab64{tab_params<double>(b->tables), b->tables->bes64},
                                                             b->ctr, b->mlp ? b->d_mout : nullptr);
    if (e1) cudaEventRecordWithFlags(e1, st, rec);
    batch_compact_head<<<(b->n_inst + 255) / 256, 256, 0, st>>>(b->d_inst, b->n_inst);
    const dim3 g(kCompactBlocks, b->n_inst);
    batch_compact_classify<<<g, 256, 0, st>>>(b->d_inst);
    batch_compact_tail<<<g, 256, 0, st>>>(b->d_inst);
    batch_compact_move<<<g, 256, 0, st>>>(b->d_inst, b->d_clk);
}

// the caller's event pair k (modulo their number), or none
static void kernel_events(const qed_batch_s* b, long long k, cudaEvent_t* e0, cudaEvent_t* e1) {
    *e0 = *e1 = nullptr;
    const long long n = (long long)b->kev.size() / 2;
    if (n == 0) return;
    const long long i = k % n;
    *e0 = b->kev[2 * i];
    *e1 = b->kev[2 * i + 1];
}

static void drop_graph(qed_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->exec_steps = 0;
}

static bool valid_instance(const qed_instance& in) {
    const qed_particles* sp[3] = {&in.electrons, &in.positrons, &in.photons};
    const int32_t charge[3] = {QED_ELECTRON, QED_POSITRON, QED_PHOTON};
    for (int k = 0; k < 3; ++k) {
        if (check_particles(sp[k], k == 2) != QED_OK || sp[k]->layout != QED_FP32 || sp[k]->charge != charge[k] ||
            sp[k]->capacity > (int64_t)INT32_MAX)  // particle indices within a buffer are 32-bit
            return false;
    }
    return valid_field(&in.field) && in.electrons.count != in.positrons.count && in.electrons.count != in.photons.count &&
           in.positrons.count != in.photons.count;
}

static inline size_t r16(size_t v) { return (v + 15) & ~size_t(15); }

extern "C" qed_status qed_batch_set_tuning(qed_batch_t b, const qed_batch_tuning* tn) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (!tn || tn->variant < 0 || tn->variant >= QED_BATCH_VARIANTS || tn->blocks_per_sm < 0 || tn->chunk < 1 ||
        tn->chunk > 4096 || tn->graph_steps < 0 || tn->graph_steps > 4096)
        return QED_ERR_ARG;
    const int occ = variant_occupancy(b, tn->variant);
    if (occ < 1) return QED_ERR_ARG;  // this variant does not fit this batch (shared memory)
    const int bps = tn->blocks_per_sm == 0 ? occ : std::min(tn->blocks_per_sm, occ);
    drop_graph(b);
    b->tuning = *tn;
    b->tuning.blocks_per_sm = bps;
    b->grid = b->sms * bps;
    return QED_OK;
}

extern "C" qed_status qed_batch_get_tuning(qed_batch_t b, qed_batch_tuning* out) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (!out) return QED_ERR_ARG;
    *out = b->tuning;
    return QED_OK;
}

extern "C" void qed_batch_destroy(qed_batch_t b) {
    if (!valid_batch(b)) return;
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_inst);
    cudaFree(b->d_seg);
    cudaFree(b->d_ctx);
    cudaFree(b->d_ev);
    cudaFree(b->d_tile0);
    cudaFree(b->d_clk);
    cudaFree(b->d_hdr);
    cudaFree(b->d_app);
    cudaFree(b->d_ws);
    cudaFree(b->d_mchi);
    cudaFree(b->d_mr);
    cudaFree(b->d_ms);
    cudaFree(b->d_mout);
    cudaFree(b->d_mlep);
    cudaFree(b->d_mfb);
    b->magic = 0;
    delete b;
}

extern "C" qed_status qed_batch_create(qed_tables_t t, const qed_instance* instances, int32_t n_inst,
                                       const qed_batch_desc* desc, qed_counters* counters_dev, qed_batch_t* out) {
    if (!out) return QED_ERR_ARG;
    *out = nullptr;
    if (!valid_tables(t)) return QED_ERR_STATE;
    if (!instances || n_inst < 1 || n_inst > QED_BATCH_MAX_INSTANCES || !desc || !counters_dev) return QED_ERR_ARG;
    if (!(desc->dt > 0.0) || !std::isfinite(desc->dt) || !std::isfinite(desc->t0) || !valid_flags(desc->flags) ||
        !(desc->photon_store_min >= 0.0) || !(desc->chi_floor >= 0.0))
        return QED_ERR_ARG;
    for (int i = 0; i < n_inst; ++i)
        if (!valid_instance(instances[i])) return QED_ERR_ARG;

    qed_batch_s* b = new qed_batch_s();
    b->magic = kBatchMagic;
    b->tables = t;
    b->n_inst = n_inst;
    b->desc = *desc;
    b->plane_waves = true;
    for (int i = 0; i < n_inst; ++i)
        b->plane_waves = b->plane_waves &&
                         (instances[i].field.kind == QED_FIELD_LP || instances[i].field.kind == QED_FIELD_CP);
    b->ctr = counters_dev;
    bool ok = cudaGetDevice(&b->device) == cudaSuccess &&
              cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess;
    // compaction scratch: per instance holes and live lists (8 B per photon of capacity each) and marks
    size_t ws = 0;
    std::vector<size_t> ws_off(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        ws_off[i] = ws;
        const size_t cap = (size_t)instances[i].photons.capacity;
        ws += 2 * r16(8 * cap) + r16(cap);
        b->capacity_total += instances[i].electrons.capacity + instances[i].positrons.capacity + instances[i].photons.capacity;
    }
    const int n_seg = kSpecies * n_inst;
    if (b->capacity_total / 32 + n_seg >= (int64_t)INT32_MAX) {  // tile indices are 32-bit
        qed_batch_destroy(b);
        return QED_ERR_ARG;
    }
    ok = ok && cudaMalloc(&b->d_inst, sizeof(InstDev) * n_inst) == cudaSuccess &&
         cudaMalloc(&b->d_seg, sizeof(SegDev) * n_seg) == cudaSuccess &&
         cudaMalloc(&b->d_ctx, sizeof(SegCtx) * n_seg) == cudaSuccess &&
         cudaMalloc(&b->d_ev, sizeof(long long) * (size_t)std::max<int64_t>(1, b->capacity_total)) == cudaSuccess &&
         cudaMalloc(&b->d_tile0, sizeof(int64_t) * (n_seg + 1)) == cudaSuccess &&
         cudaMalloc(&b->d_clk, sizeof(ClockDev)) == cudaSuccess &&
         cudaMalloc(&b->d_hdr, sizeof(int64_t) * 4 * n_inst) == cudaSuccess &&
         cudaMalloc(&b->d_app, sizeof(AppendState) * 2 * n_inst) == cudaSuccess &&
         cudaMalloc(&b->d_ws, ws < 16 ? 16 : ws) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        qed_batch_destroy(b);
        return QED_ERR_NOMEM;
    }
    std::vector<InstDev> h(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        const qed_instance& in = instances[i];
        InstDev& d = h[i];
        d.F = field_params<float>(in.field);
        d.F64 = field_params<double>(in.field);
        d.phase = in.field.phase;
        d.seed = in.seed;
        d.sp[0] = part_dev(&in.electrons);
        d.sp[1] = part_dev(&in.positrons);
        d.sp[2] = part_dev(&in.photons);
        const size_t cap = (size_t)in.photons.capacity;
        unsigned char* base = b->d_ws + ws_off[i];
        d.holes = (int64_t*)base;
        d.live = (int64_t*)(base + r16(8 * cap));
        d.mark = base + 2 * r16(8 * cap);
        d.hdr = b->d_hdr + 4 * i;
        d.app = b->d_app + 2 * i;
    }
    ClockDev clk{};
    clk.step = desc->step0;
    clk.step0 = desc->step0;
    clk.t0 = desc->t0;
    clk.dt = desc->dt;
    ok = cudaMemcpy(b->d_inst, h.data(), sizeof(InstDev) * n_inst, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_clk, &clk, sizeof(ClockDev), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(b->d_ws, 0, ws < 16 ? 16 : ws) == cudaSuccess &&
         cudaMemset(b->d_hdr, 0, sizeof(int64_t) * 4 * n_inst) == cudaSuccess &&
         cudaMemset(b->d_app, 0, sizeof(AppendState) * 2 * n_inst) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        qed_batch_destroy(b);
        return QED_ERR_CUDA;
    }
    int ev_per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ev_per_sm, batch_event_kernel, kEventThreads, 0);
    b->ev_grid = b->sms * std::max(1, ev_per_sm);
    const qed_batch_tuning def{0, 0, 64, 8};
    if (qed_batch_set_tuning(b, &def) != QED_OK) {
        qed_batch_destroy(b);
        return QED_ERR_CUDA;
    }
    *out = b;
    return QED_OK;
}

extern "C" qed_status qed_batch_step(qed_batch_t b, int32_t n_steps, void* stream) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (n_steps < 0) return QED_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int done = 0;
    const int G = b->tuning.graph_steps;
    if (G > 0 && (n_steps >= G || n_steps == 0)) {
        if (!b->exec) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return QED_ERR_CUDA;
            for (int k = 0; k < G; ++k) {
                cudaEvent_t e0, e1;
                kernel_events(b, k, &e0, &e1);
                launch_batch_step(b, b->cap_stream, e0, e1, true);
            }
            const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
            if (e != cudaSuccess || !g) {
                cudaGetLastError();
                return QED_ERR_CUDA;
            }
            const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                b->exec = nullptr;
                cudaGetLastError();
                return QED_ERR_CUDA;
            }
            b->exec_steps = G;
        }
        for (; done + G <= n_steps; done += G)
            if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return QED_ERR_CUDA;
    }
    for (; done < n_steps; ++done) {
        cudaEvent_t e0, e1;
        kernel_events(b, b->direct_steps++, &e0, &e1);
        launch_batch_step(b, st, e0, e1);
    }
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_batch_set_kernel_events(qed_batch_t b, void* const* events, int32_t n_pairs) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (n_pairs < 0 || n_pairs > (1 << 20) || (n_pairs > 0 && !events)) return QED_ERR_ARG;
    for (int32_t i = 0; i < 2 * n_pairs; ++i)
        if (!events[i]) return QED_ERR_ARG;
    drop_graph(b);
    b->kev.assign((cudaEvent_t*)events, (cudaEvent_t*)events + 2 * n_pairs);
    b->direct_steps = 0;
    return QED_OK;
}

extern "C" qed_status qed_batch_set_mlp(qed_batch_t b, qed_mlp_t m, double tol) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (m && !mlp_valid(m)) return QED_ERR_STATE;
    if (m && (!(tol > 0.0) || !(tol < 1.0) || (b->desc.flags & QED_F_REJECT))) return QED_ERR_ARG;
    drop_graph(b);
    if (!m) {
        b->mlp = nullptr;
        return QED_OK;
    }
    if (!b->d_mout) {
        const size_t n = (size_t)std::max<int64_t>(1, b->capacity_total);
        const bool ok = cudaMalloc(&b->d_mchi, 8 * n) == cudaSuccess && cudaMalloc(&b->d_mr, 8 * n) == cudaSuccess &&
                        cudaMalloc(&b->d_ms, 8 * n) == cudaSuccess && cudaMalloc(&b->d_mout, 16 * n) == cudaSuccess &&
                        cudaMalloc(&b->d_mlep, n) == cudaSuccess &&
                        cudaMalloc(&b->d_mfb, sizeof(unsigned long long)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            cudaFree(b->d_mchi);
            cudaFree(b->d_mr);
            cudaFree(b->d_ms);
            cudaFree(b->d_mout);
            cudaFree(b->d_mlep);
            cudaFree(b->d_mfb);
            b->d_mchi = b->d_mr = b->d_ms = nullptr;
            b->d_mout = nullptr;
            b->d_mlep = nullptr;
            b->d_mfb = nullptr;
            return QED_ERR_NOMEM;
        }
    }
    if (cudaMemset(b->d_mfb, 0, sizeof(unsigned long long)) != cudaSuccess) return QED_ERR_CUDA;
    b->mlp = m;
    b->mlp_tol = tol;
    b->mlp_grid = mlp_listed_grid(std::max<int64_t>(1, b->capacity_total));
    return QED_OK;
}

extern "C" qed_status qed_batch_mlp_last(qed_batch_t b, int64_t n_max, double* chi, double* r, double* s_beta,
                                         float* out4, uint8_t* is_lepton, int64_t* n_out,
                                         unsigned long long* n_fallback_total) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (!b->d_mout) return QED_ERR_STATE;  // no network was ever set
    if (n_max < 0) return QED_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return QED_ERR_CUDA;
    ClockDev clk;
    unsigned long long fb = 0;
    if (cudaMemcpy(&clk, b->d_clk, sizeof(ClockDev), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&fb, b->d_mfb, sizeof(fb), cudaMemcpyDeviceToHost) != cudaSuccess)
        return QED_ERR_CUDA;
    if (n_out) *n_out = (int64_t)clk.n_events;
    if (n_fallback_total) *n_fallback_total = fb;
    const size_t n = (size_t)std::min<int64_t>(n_max, (int64_t)clk.n_events);
    if (n == 0) return QED_OK;
    bool ok = true;
    if (chi) ok = ok && cudaMemcpy(chi, b->d_mchi, 8 * n, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (r) ok = ok && cudaMemcpy(r, b->d_mr, 8 * n, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (s_beta) ok = ok && cudaMemcpy(s_beta, b->d_ms, 8 * n, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (out4) ok = ok && cudaMemcpy(out4, b->d_mout, 16 * n, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (is_lepton) ok = ok && cudaMemcpy(is_lepton, b->d_mlep, n, cudaMemcpyDeviceToHost) == cudaSuccess;
    return ok ? QED_OK : QED_ERR_CUDA;
}

extern "C" qed_status qed_batch_stats_read(qed_batch_t b, qed_batch_stats* out, void* stream) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (!out) return QED_ERR_ARG;
    ClockDev c;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&c, b->d_clk, sizeof(ClockDev), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QED_ERR_CUDA;
    out->step = c.step;
    out->particle_steps = c.psteps;
    for (int k = 0; k < kSpecies; ++k) {
        out->species_steps[k] = c.species_steps[k];
        out->alive[k] = c.alive[k];
    }
    return QED_OK;
}

// ---- autotuner ------------------------------------------------------------------------------------
static std::string tune_key(const qed_batch_s* b) {
    cudaDeviceProp p;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&p, b->device) == cudaSuccess) name = p.name;
    for (char& ch : name)
        if (ch == ' ' || ch == '"' || ch == '\\') ch = '_';
    int lg = 0;
    while (lg < 62 && (1ll << (lg + 1)) <= b->capacity_total) ++lg;
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d|inst%d|cap2^%d|nchi%d", name.c_str(), b->sms, b->n_inst, lg, b->tables->desc.n_chi);
    return buf;
}

static bool json_int(const char* line, const char* field, int* v) {
    char pat[64];
    snprintf(pat, sizeof pat, "\"%s\": ", field);
    const char* p = strstr(line, pat);
    return p && sscanf(p + strlen(pat), "%d", v) == 1;
}

static bool cache_lookup(const char* path, const std::string& key, qed_batch_tuning* tn) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    const std::string pat = "\"key\": \"" + key + "\"";
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        if (!strstr(line, pat.c_str())) continue;
        int v, bps, ch;
        if (json_int(line, "variant", &v) && json_int(line, "blocks_per_sm", &bps) && json_int(line, "chunk", &ch)) {
            tn->variant = v;
            tn->blocks_per_sm = bps;
            tn->chunk = ch;
            found = true;  // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

extern "C" qed_status qed_batch_tune(qed_batch_t b, int32_t steps_per_candidate, const char* cache_path,
                                     qed_batch_tuning* out, void* stream) {
    if (!valid_batch(b)) return QED_ERR_STATE;
    if (steps_per_candidate < 1 || steps_per_candidate > 1000) return QED_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int graph_steps = b->tuning.graph_steps;
    const std::string key = tune_key(b);
    qed_batch_tuning best = b->tuning;
    if (cache_path && cache_lookup(cache_path, key, &best)) {
        best.graph_steps = graph_steps;
        const qed_status s = qed_batch_set_tuning(b, &best);
        if (s == QED_OK) {
            if (out) *out = b->tuning;
            return QED_OK;
        }
    }
    // candidates: every variant that fits, at its occupancy maximum and one block fewer, with the longest
    // runs of the guided schedule capped at 32, 64 or 128 tiles
    std::vector<qed_batch_tuning> cand;
    for (int v = 0; v < QED_BATCH_VARIANTS; ++v) {
        const int occ = variant_occupancy(b, v);
        for (int bps = occ; bps >= 1 && bps >= occ - 1; --bps)
            for (int ch : {32, 64, 128}) cand.push_back(qed_batch_tuning{v, bps, ch, 0});
    }
    if (cand.empty()) return QED_ERR_CUDA;
    std::vector<double> score(cand.size(), 1e300);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QED_ERR_CUDA;
    qed_status status = QED_OK;
    for (int pass = 0; pass < 2 && status == QED_OK; ++pass) {
        for (size_t c = 0; c < cand.size() && status == QED_OK; ++c) {
            const size_t k = pass == 0 ? c : cand.size() - 1 - c;  // second pass in reverse: drift cancels
            if (qed_batch_set_tuning(b, &cand[k]) != QED_OK) continue;
            qed_batch_stats s0, s1;
            if (qed_batch_stats_read(b, &s0, stream) != QED_OK) {
                status = QED_ERR_CUDA;
                break;
            }
            double ms = 0.0;
            for (int r = 0; r < steps_per_candidate; ++r) {
                launch_batch_step(b, st, e0, e1);
                float x = 0.0f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&x, e0, e1) != cudaSuccess) {
                    status = QED_ERR_CUDA;
                    break;
                }
                ms += x;
            }
            if (status != QED_OK || qed_batch_stats_read(b, &s1, stream) != QED_OK) {
                status = QED_ERR_CUDA;
                break;
            }
            const double ps = (double)(s1.particle_steps - s0.particle_steps);
            if (ps > 0) score[k] = std::min(score[k], ms * 1e6 / ps);  // ns per particle-step
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != QED_OK) return status;
    size_t bi = 0;
    for (size_t c = 1; c < cand.size(); ++c)
        if (score[c] < score[bi]) bi = c;
    best = cand[bi];
    best.graph_steps = graph_steps;
    const qed_status s = qed_batch_set_tuning(b, &best);
    if (s != QED_OK) return s;
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "{\"key\": \"%s\", \"variant\": %d, \"blocks_per_sm\": %d, \"chunk\": %d, \"ns_per_particle_step\": %.6g}\n",
                    key.c_str(), best.variant, best.blocks_per_sm, best.chunk, score[bi]);
            fclose(f);
        }
    }
    if (out) *out = b->tuning;
    return QED_OK;
}
