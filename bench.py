"""Throughput of the spin/polarization-resolved QED step on GB300.

Workload (default, --workload batched): 96 independent collisions stepped together, N_i log-uniform in
[1e3, 2e6] electrons (2.2e7 in all), a0 ~ U[10, 300], gamma ~ U[500, 8000], partially polarized spins
(+-n_i, P(+) = (1 + d_i)/2), LP and CP alternating, 0.8 um, 10-cycle sin^2 envelopes, NLC + NBW,
daughters appended to per-instance buffers of 4x the initial count, dt = lambda/(100 c), FP32 path with
FP64 optical depth.  One step of the batch = the planning kernel, one persistent kernel over every
instance and species, and the per-instance photon compaction, replayed from a CUDA graph; the launch
shape comes from the library's autotuner (timed on the run's own steps during the untimed advance).
The batch is advanced (untimed) into the interaction, then W warm-up steps and K timed steps run as
one graph launch; particle-steps are the photons, electrons and positrons alive at each step's start,
counted on the device.  The particle state (several GB) is far larger than L2: no flush is needed.

--workload headon: the single-buffer entry points on one collision (1e7 electrons, gamma 4000, spin +z,
CP a0 = 150, 20 cycles).

--workload helicity: the plane-wave analogues of the helicity-transfer benchmarks (10 GeV electrons of
helicity +1 against an LP a0 = 50 pulse and a CP a0 = 100 pulse, 1e6 electrons each, two instances of one
batch), the whole crossing timed, with the photons' circular polarization and the positrons' longitudinal
polarization against energy.

--workload cascade: 2e8 electrons (gamma 1000) where two CP pulses (a0 = 500, 1 um, 15 cycles) collide,
the whole 3000-step run through the batched path as one instance: the pair cascade multiplies the
leptons, compaction every step; photons below 300 m c^2 are not stored.  Timed: all 3000 steps, in
graph launches of 500 steps; the error leg runs three extra (untimed) steps after step 1000.

Multi-GPU (torchrun): every rank runs an independent replica with its own seeds (particles never
interact across ranks; there is no data-path collective): weak scaling.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload batched|headon]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QED particle-steps/s on 1 GB300 (FP32 batched vs plain FP64) at stated error; % HBM peak"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="batched", choices=["batched", "headon", "cascade", "helicity"])
    ap.add_argument("--electrons", type=int, default=10_000_000, help="headon workload only")
    ap.add_argument("--advance", type=int, default=None,
                    help="untimed steps before warm-up (into the interaction; default 450 batched, 620 headon)")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, e2e and CPU-baseline legs")
    ap.add_argument("--no-tune", action="store_true", help="batched: keep the default launch shape")
    ap.add_argument("--tuning", default=None,
                    help="batched: fixed launch shape 'variant,blocks_per_sm,chunk' instead of the autotuner")
    ap.add_argument("--no-mlp", action="store_true", help="skip the learned-sampler leg")
    ap.add_argument("--no-headon", action="store_true", help="batched: skip the config-2 head-on leg")
    ap.add_argument("--cascade-steps", type=int, default=None, help="cascade: steps of the run (default 3000)")
    ap.add_argument("--flags", default="full", choices=["full", "reject"],
                    help="batched: the full flag set, or with the table-free rejection sampler (QED_F_REJECT)")
    ap.add_argument("--mlp-train", type=float, default=5e7, help="learned sampler: training samples")
    ap.add_argument("--mlp-eval", type=float, default=1e8, help="learned sampler: evaluated events")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="batched: multiply every instance's electron count (small cases for profiling)")
    a = ap.parse_args()
    if a.advance is None:
        a.advance = 450 if a.workload == "batched" else 620
    return a


# ------------------------------------------------------------------------------------------------
def clocks_sampler(stop, out, index=0):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                              "-i", str(index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return
    def reader():
        for line in p.stdout:
            out.append(line.strip())
    t = threading.Thread(target=reader, daemon=True)
    t.start()
    stop.wait()
    p.terminate()
    try:
        p.wait(timeout=2)
    except Exception:
        p.kill()
    t.join(timeout=2)


def summarize_clocks(lines):
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = max(mx, float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = ("qed_batch.cu", "qed_step32.cuh", "qed_device.cuh", "qed_bessel.cuh", "qed_steps.h", "qed_internal.h")


def kernel_source_hash() -> str:
    """sha256 over the code of the sources the batched kernels are built from: `//` comments and blank
    lines are left out, so a change of wording keeps a capture of the same kernels valid."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_08929_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes per particle-step of the batched kernel from the committed ncu summary, if it was taken
    on the kernel as it is now (same source hash); else None."""
    p = os.path.join(ROOT, "profiles", "batch_step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d if d.get("source_sha256") == kernel_source_hash() else None


# Algorithmic bytes of the FP32 particle traffic, the roofline's numerator.  The per-unit figures the
# roofline is quoted on: a lepton-step moves 96 B (read x, p, s 36 + tau 8 + id 8; write x, p, s, tau 44),
# a photon-step 84 B (read x, k, P 36 + tau 8 + id 8; write x, P, tau 32), a stored daughter 52 B.  The
# smaller figures this layout needs (reported beside them): 88 B per lepton-step (the id only at events,
# 8 B per event), 56 B per photon-step (read 44, write x 12) + 20 B (P, tau) for a photon with a pair
# rate; 52 B per stored daughter.
def unit_bytes(lepton_steps, photon_steps, stored):
    return 96.0 * lepton_steps + 84.0 * photon_steps + 52.0 * stored


def design_bytes(lepton_steps, photon_steps, rate_steps, events, stored):
    return 88.0 * lepton_steps + 56.0 * photon_steps + 20.0 * rate_steps + 8.0 * events + 52.0 * stored


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------------
class Sim:
    """The three species on the device and one full QED time step through the C ABI."""

    def __init__(self, Q, B, I, wl, layout, tables, n, seed, caps, device):
        """caps: (electron, positron, photon) capacities"""
        import torch
        self.Q, self.B, self.torch = Q, B, torch
        self.wl = wl
        self.tables = tables
        self.field = Q.laser_field(wl.laser)
        self.el = Q.ParticleBuffer(caps[0], layout, B.QED_ELECTRON, device=device, use_begin=True)
        self.po = Q.ParticleBuffer(caps[1], layout, B.QED_POSITRON, device=device, use_begin=True)
        self.ph = Q.ParticleBuffer(caps[2], layout, B.QED_PHOTON, device=device, photons=True, use_begin=True)
        self.ws = Q.CompactWorkspace(caps[2], device=device)
        self.ctr = Q.Counters(device=device)
        self.seed = seed
        self.n0 = n
        self.step_index = 0
        self.stream = torch.cuda.current_stream().cuda_stream

    def load_beam(self, beam):
        beam = z_order(beam)
        self.el.load(beam["pos"], beam["mom"], beam["spin"], beam["w"], beam["id"])
        self.el.init_tau(self.seed)

    def load_state(self, st):
        for buf, key in ((self.el, "el"), (self.po, "po"), (self.ph, "ph")):
            d = st[key]
            buf.load(d["pos"], d["mom"], d["spin"], d["w"], d["id"], tau=d["tau"])

    def state(self):
        return {"el": self.el.read(), "po": self.po.read(), "ph": self.ph.read()}

    def step(self, kernel_events=None):
        B, Q = self.B, self.Q
        s = self.step_index
        st = Q.step_desc(self.wl.dt, s * self.wl.dt, s, self.seed, B.QED_F_FULL, self.wl.photon_store_min)
        B.qed_snapshot_counts([self.el.s, self.po.s, self.ph.s], self.stream)
        ev = kernel_events
        if ev is not None:
            ev["pair"][0].record()
        B.qed_pair_step(self.tables.handle, self.field, st, self.ph.s, self.el.s, self.po.s, self.ctr.ptr, self.stream)
        if ev is not None:
            ev["pair"][1].record()
            ev["push"][0].record()
        B.qed_push_step(self.tables.handle, self.field, st, self.el.s, self.ph.s, self.ctr.ptr, self.stream)
        if ev is not None:
            ev["push"][1].record()
        B.qed_push_step(self.tables.handle, self.field, st, self.po.s, self.ph.s, self.ctr.ptr, self.stream)
        B.qed_compact(self.ph.s, self.ws.ptr, self.ws.bytes, self.stream)
        self.step_index += 1

    LAUNCHES_PER_STEP = 11  # snapshot 1, pair 2, push 2 x 2, compaction 4

    def begins(self):
        return self.torch.stack([self.el.counts[1], self.po.counts[1], self.ph.counts[1]])


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args) if args.workload == "headon" else reference_arm_batch(args)
    run = {"headon": native, "cascade": native_cascade, "helicity": native_helicity}.get(args.workload, native_batch)
    out = run(args)
    if out is not None:
        print(json.dumps(out))


# ------------------------------------------------------------------------------------------------
def native(args):
    import torch
    from paper_2511_08929_gb300 import binding as B
    from paper_2511_08929_gb300 import build as bld
    from paper_2511_08929_gb300 import buffers as Q
    from paper_2511_08929_gb300 import inputs as I

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = f"cuda:{local if world > 1 else 0}"
    bld.build()
    wl = I.HEADON_CP_LARGE
    n = args.electrons
    seed = wl.seed + 1000 * rank
    t0 = time.time()
    tables = Q.Tables(1e-4, 1e3, wl.n_chi, wl.n_r)
    torch.cuda.synchronize()
    t_tables = time.time() - t0
    beam = I.lepton_beam(n, wl.gamma, direction=(0.0, 0.0, -1.0), z_range=(2 * math.pi, 22 * math.pi),
                         spin="fixed", spin_dir=(0.0, 0.0, 1.0), seed=seed, id_offset=rank * (1 << 40))
    # buffers from a measured growth curve: a 1/64 subsample stepped through the whole run with roomy
    # buffers, then margin 1.25 (the configuration's 4x the initial count drops most daughters by then)
    end_step = args.advance + args.warmup + args.steps + 16
    sub = _subsample(beam, max(256, n // 64))
    m = len(sub["id"])
    probe = Sim(Q, B, I, wl, B.QED_FP32, tables, m, seed, (8 * m + 4096, 8 * m + 4096, 400 * m + 4096), device)
    probe.load_beam(sub)
    peak = np.zeros(3)
    for _ in range(end_step):
        probe.step()
        if probe.step_index % 25 == 0 or probe.step_index == end_step:
            peak = np.maximum(peak, torch.stack([probe.el.counts[0], probe.po.counts[0], probe.ph.counts[0]]).cpu().numpy())
    if probe.ctr.read().status != 0:
        raise SystemExit("bench: the buffer sizing pass overflowed")
    caps = tuple(int(1.25 * peak[i] / m * n) + 4096 for i in range(3))
    del probe
    torch.cuda.empty_cache()
    sim = Sim(Q, B, I, wl, B.QED_FP32, tables, n, seed, caps, device)
    sim.load_beam(beam)
    for _ in range(args.advance):
        sim.step()
    for _ in range(args.warmup):
        sim.step()
    torch.cuda.synchronize()

    K = args.steps
    hist = torch.zeros((K, 3), dtype=torch.int64, device=device)
    evs = [{k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in ("pair", "push")}
           for _ in range(K)]
    sim.ctr.zero()
    stop = threading.Event()
    clock_lines = []
    th = threading.Thread(target=clocks_sampler, args=(stop, clock_lines, local), daemon=True)
    th.start()
    time.sleep(0.5)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for k in range(K):
        hist[k].copy_(torch.stack([sim.el.counts[0], sim.po.counts[0], sim.ph.counts[0]]))  # alive at step start
        sim.step(kernel_events=evs[k])
    end.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stop.set()
    th.join(timeout=5)
    ms = start.elapsed_time(end)
    t_pair = sum(e["pair"][0].elapsed_time(e["pair"][1]) for e in evs)
    t_push = sum(e["push"][0].elapsed_time(e["push"][1]) for e in evs)
    ctr = sim.ctr.read()
    if ctr.status != 0:
        raise SystemExit(f"bench: the timed steps ended with status {ctr.status} ({B.status_string(ctr.status)}), "
                         f"{ctr.dropped_capacity} daughters dropped: no valid measurement")
    h = hist.cpu().numpy().astype(np.float64)
    psteps = float(h.sum())
    n_el, n_po, n_ph = h[:, 0].sum(), h[:, 1].sum(), h[:, 2].sum()
    tmax = ms
    psteps_all = psteps
    if dist is not None:
        tmax, psteps_all = reduce_over_ranks(ms, psteps, dist, device)
    value = psteps_all / (tmax / 1e3)

    # roofline of the dominant kernel: algorithmic bytes per launch / its event-timed duration (the
    # per-unit figures of unit_bytes; the stored daughters of all species are counted with both kernels,
    # an upper bound)
    peak, peak_kind = measured_peaks()
    push_bytes = unit_bytes(n_el + n_po, 0.0, ctr.stored)
    pair_bytes = unit_bytes(0.0, n_ph, ctr.stored)
    bw_push = push_bytes / (t_push / 1e3) / 1e9 if t_push > 0 else 0.0
    bw_pair = pair_bytes / (t_pair / 1e3) / 1e9 if t_pair > 0 else 0.0
    dominant = "photon_step" if t_pair >= t_push else "electron_step"
    achieved = bw_pair if t_pair >= t_push else bw_push
    roof = {"kernel": dominant, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_kind,
            "electron_step": {"GBps": round(bw_push, 1), "ms_per_launch": round(t_push / K, 4),
                              "algorithmic_bytes_per_launch": push_bytes / K},
            "photon_step": {"GBps": round(bw_pair, 1), "ms_per_launch": round(t_pair / K, 4),
                            "algorithmic_bytes_per_launch": pair_bytes / K}}
    clocks = summarize_clocks(clock_lines)

    extras = {}
    if not args.no_extras and rank == 0:
        extras = extra_legs(args, sim, Q, B, I, wl, tables, device, torch)
    elif getattr(args, "fp64_leg", False) and rank == 0:
        extras = extra_legs(args, sim, Q, B, I, wl, tables, device, torch, legs=("fp64",))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": tmax / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "electrons_per_gpu": n, "gamma": wl.gamma, "a0": wl.laser.a0,
                   "laser": "CP 0.8um 20 cycles", "buffers": f"sized from a measured growth curve {list(caps)}",
                   "layout": "FP32 float4 SoA",
                   "timed_from_step": args.advance + args.warmup, "parallelism": f"replicas x{world}",
                   "l2": "state > L2 (no flush needed)", "tables": "256 chi x 256 r, FP64-built"},
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": Sim.LAUNCHES_PER_STEP * K,
        "particles_at_start": {"electrons": int(h[0, 0]), "positrons": int(h[0, 1]), "photons": int(h[0, 2])},
        "counters": {k: int(v) for k, v in ctr.as_dict().items()},
        "table_build_s": round(t_tables, 2),
    }
    out.update(extras)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return None
    return out


# ------------------------------------------------------------------------------------------------
# the batched workload
# ------------------------------------------------------------------------------------------------
def z_order(beam: dict) -> dict:
    """The same particles (each keeps its id and state) laid out in memory by position along the beam
    axis, so that the 32 particles of a tile enter and leave the pulse together."""
    o = np.argsort(beam["pos"][:, 2], kind="stable")
    return {k: v[o] for k, v in beam.items()}


def reduce_over_ranks(ms: float, psteps: float, dist, device):
    """Whole-job timing of independent replicas: the slowest rank's time and every rank's particle-steps."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([psteps], dtype=torch.float64, device=device)
    dist.all_reduce(p)
    return float(t.item()), float(p.item())


def replica_plan(wl, rank: int):
    """Rank `rank`'s replica of a batched workload: the same instances, Philox seeds offset by 1000 rank
    and particle ids by rank 2^48, so that no two ranks share a key (the replicas are independent)."""
    insts = wl.instances()
    seeds = [x["seed"] + 1000 * rank for x in insts]
    return insts, seeds, np.uint64(rank << 48)


def batch_workload(I, scale=1.0):
    import dataclasses
    wl = I.BATCHED_96
    if scale != 1.0:
        wl = dataclasses.replace(wl, name=f"{wl.name}_x{scale:g}", n_min=wl.n_min * scale, n_max=wl.n_max * scale)
    return wl


def _subsample(beam: dict, m: int) -> dict:
    """m particles spread evenly over the beam's id order (ids are drawn independently of position)."""
    n = len(beam["id"])
    if m >= n:
        return beam
    ix = np.linspace(0, n - 1, m).round().astype(np.int64)
    return {k: v[ix] for k, v in beam.items()}


def growth_capacities(Q, B, tables, wl, insts, fields, seeds, end_step, device, sub=64, min_sub=256, margin=1.25,
                      flags=None):
    """Buffer capacities from a measured growth curve.  A strided subsample of every instance (1/sub of
    its electrons, at least min_sub) is stepped on the GPU through end_step steps with generous buffers,
    and each species' largest count per initial electron is recorded; the batch then gets
    margin x that x N_i + 4096 slots per species and instance.  Particles never interact, so the growth
    per initial electron of a subsample is that of the whole beam up to sampling noise (the margin)."""
    import torch
    fac = [8.0, 8.0, 400.0]
    for _attempt in range(3):
        subs = [wl.sample(k, x, min(x["n"], max(min_sub, x["n"] // sub))) if hasattr(wl, "sample") else
                _subsample(wl.beam(k, x), min(x["n"], max(min_sub, x["n"] // sub))) for k, x in enumerate(insts)]
        caps = [tuple(max(4096, int(f * len(b["id"]))) for f in fac) for b in subs]
        bt = Q.Batch(tables, fields, seeds, caps, wl.dt, t0=0.0, step0=0, photon_store_min=wl.photon_store_min,
                     device=device, flags=flags)
        bt.set_tuning(0, 0, 16, 25)
        for k, ((e, _, _), b) in enumerate(zip(bt.buffers(), subs)):
            b = z_order(b)
            e.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
            e.init_tau(seeds[k])
        peak = np.zeros((len(insts), 3))
        done = 0
        while done < end_step:
            n = min(25, end_step - done)
            bt.step(n)
            done += n
            cnt = torch.stack([b.counts[0] for x in bt.buffers() for b in x]).cpu().numpy().reshape(-1, 3)
            peak = np.maximum(peak, cnt)
        status = bt.ctr.read().status
        bt.close()
        torch.cuda.empty_cache()
        if status == 0:
            per = peak / np.array([len(b["id"]) for b in subs], dtype=np.float64)[:, None]
            out = [tuple(int(margin * per[k, s] * x["n"]) + 4096 for s in range(3)) for k, x in enumerate(insts)]
            return out, {"subsample": f"1/{sub} of each instance's electrons (at least {min_sub})",
                         "steps": int(end_step), "margin": margin,
                         "photons_per_electron_max": float(per[:, 2].max()),
                         "slots": int(sum(sum(c) for c in out))}
        fac = [2 * f for f in fac]
    raise RuntimeError("buffer sizing pass overflowed three times")


def batch_setup(Q, B, I, tables, rank, device, scale=1.0, caps=None, flags=None):
    wl = batch_workload(I, scale)
    insts, seeds, id_offset = replica_plan(wl, rank)
    fields = [Q.laser_field(wl.laser(x)) for x in insts]
    if caps is None:
        caps = [tuple(max(4096, int(wl.capacity_factor * x["n"])) for _ in range(3)) for x in insts]
    bt = Q.Batch(tables, fields, seeds, caps, wl.dt, t0=0.0, step0=0, photon_store_min=wl.photon_store_min,
                 device=device, flags=flags)
    for k, (x, (e, p, g)) in enumerate(zip(insts, bt.buffers())):
        b = z_order(wl.beam(k, x))
        b["id"] = b["id"] + id_offset
        e.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
        e.init_tau(seeds[k])
    return wl, insts, fields, seeds, caps, bt


def native_batch(args):
    import torch
    from paper_2511_08929_gb300 import binding as B
    from paper_2511_08929_gb300 import build as bld
    from paper_2511_08929_gb300 import buffers as Q
    from paper_2511_08929_gb300 import inputs as I

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = f"cuda:{local if world > 1 else 0}"
    bld.build()
    t0 = time.time()
    tables = Q.Tables(1e-4, 1e3, 256, 256)
    torch.cuda.synchronize()
    t_tables = time.time() - t0
    extras_on = not args.no_extras and rank == 0
    E2E_STEPS, ERR_STEPS = 3, 3
    MLP_STEPS = 4 * MLP_WINDOW if extras_on and not args.no_mlp and args.flags == "full" else 0
    # every step the run takes on the FP32 batch: advance, warm-up, e2e, timed, error legs, the learned
    # sampler's windows (+ slack)
    end_step = args.advance + args.warmup + (E2E_STEPS if extras_on else 0) + args.steps + \
        (ERR_STEPS if extras_on else 0) + MLP_STEPS + 16
    wl0 = batch_workload(I, args.scale)
    insts0, seeds0, _ = replica_plan(wl0, rank)
    fields0 = [Q.laser_field(wl0.laser(x)) for x in insts0]
    t0 = time.time()
    flags = {"full": None, "reject": B.QED_F_FULL | B.QED_F_REJECT}[args.flags]
    caps, sizing = growth_capacities(Q, B, tables, wl0, insts0, fields0, seeds0, end_step, device, flags=flags)
    sizing["seconds"] = round(time.time() - t0, 2)
    wl, insts, fields, seeds, caps, bt = batch_setup(Q, B, I, tables, rank, device, args.scale, caps=caps, flags=flags)
    stream = torch.cuda.current_stream().cuda_stream

    # untimed advance into the interaction; the autotuner times its candidates on real steps near its end
    # (about 180 steps: up to 30 shapes, two passes, three steps each), where the particle populations
    # are closest to those of the timed steps
    pre = max(0, args.advance - 180)
    bt.step(pre, stream)
    tuning = bt.tuning()
    tune_s = 0.0
    if args.tuning:
        v, bps, ch = (int(x) for x in args.tuning.split(","))
        bt.set_tuning(v, bps, ch, tuning.graph_steps)
        tuning = bt.tuning()
    elif not args.no_tune:
        cache = os.environ.get("QED_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "qedgb",
                                                              "autotune.jsonl"))
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        t0 = time.time()
        tuning = bt.tune(3, cache, stream)  # 3 steps per candidate and pass: less noise than one
        tune_s = time.time() - t0
    st = bt.stats(stream)
    if st.step < args.advance:
        bt.step(int(args.advance - st.step), stream)
    bt.step(args.warmup, stream)
    torch.cuda.synchronize()

    extras = {}
    if extras_on:  # end to end through the C ABI with host-resident state (3 steps, just before the timed ones)
        extras["e2e"] = e2e_leg(bt, torch, E2E_STEPS)

    # the timed region is one launch of a graph of K steps with event pairs around each persistent kernel
    K = args.steps
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    B.qed_batch_set_tuning(bt.handle, B.QedBatchTuning(tuning.variant, tuning.blocks_per_sm, tuning.chunk, K))
    bt.set_kernel_events(kev)
    bt.step(0, stream)  # capture and instantiate outside the timed region
    bt.ctr.zero()
    torch.cuda.synchronize()
    s0 = bt.stats(stream)
    stop = threading.Event()
    clock_lines = []
    th = threading.Thread(target=clocks_sampler, args=(stop, clock_lines, local), daemon=True)
    th.start()
    time.sleep(0.5)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    bt.step(K, stream)
    end.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stop.set()
    th.join(timeout=5)
    ms = start.elapsed_time(end)
    s1 = bt.stats(stream)
    ctr = bt.ctr.read()
    if ctr.status != 0:  # a window with dropped daughters or skipped particles did less than the step's work
        raise SystemExit(f"bench: the timed steps ended with status {ctr.status} ({B.status_string(ctr.status)}), "
                         f"{ctr.dropped_capacity} daughters dropped: no valid measurement")
    try:
        t_kern = [a.elapsed_time(b) for a, b in kev]
    except RuntimeError:
        t_kern = None
    psteps = float(s1.particle_steps - s0.particle_steps)
    d_sp = [float(s1.species_steps[i] - s0.species_steps[i]) for i in range(3)]
    tmax, psteps_all = ms, psteps
    if dist is not None:
        tmax, psteps_all = reduce_over_ranks(ms, psteps, dist, device)
    value = psteps_all / (tmax / 1e3)

    # roofline of the persistent kernel: algorithmic bytes per launch / its event-timed duration
    peak, peak_kind = measured_peaks()
    alg = unit_bytes(d_sp[0] + d_sp[1], d_sp[2], ctr.stored)
    alg_design = design_bytes(d_sp[0] + d_sp[1], d_sp[2], ctr.rate_steps, ctr.events, ctr.stored)
    tr = measured_traffic()
    traffic = None
    if tr is not None:  # ncu DRAM bytes per particle-step of a smaller capture, scaled to this launch
        traffic = tr["dram_bytes_per_particle_step"] * psteps / K
    # the timed span of a step: the persistent streaming kernel and the event kernel that follows it
    roof = {"kernel": "batch_step_kernel+batch_event_kernel", "bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s",
            "frac": None, "traffic": traffic, "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": alg / K, "design_bytes_per_launch": alg_design / K}
    if tr is not None:
        roof["traffic_source"] = tr["source"]
    if t_kern:
        tk = sum(t_kern)
        achieved = alg / (tk / 1e3) / 1e9
        roof.update({"achieved": round(achieved, 1), "frac": round(achieved / peak, 4),
                     "frac_design_bytes": round(alg_design / (tk / 1e3) / 1e9 / peak, 4),
                     "ms_per_launch": round(tk / K, 4), "share_of_step": round(tk / ms, 4)})
    clocks = summarize_clocks(clock_lines)
    if extras_on:
        err, cpu = error_leg(bt, wl, fields, seeds, torch, ERR_STEPS)
        extras["error"] = err
        extras["cpu_baseline"] = cpu
        extras["fp64_plain"] = fp64_leg(bt, wl, fields, seeds, tables, Q, B, torch, stream)
    if extras_on and not args.no_mlp:
        extras["mlp"] = mlp_leg(args, tables, torch, bt if MLP_STEPS else None, stream)
        bt.close()
        torch.cuda.empty_cache()
    if extras_on and not args.no_headon:
        bt.close()
        torch.cuda.empty_cache()
        extras["config2_headon"] = headon_leg(args)
    n_el = sum(x["n"] for x in insts)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": tmax / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name + ("" if args.flags == "full" else "_reject"), "instances": len(insts),
                   "electrons_per_gpu": n_el, "flags": args.flags,
                   "laser": "LP/CP alternating 0.8um 10 cycles, a0 U[10,300]", "gamma": "U[500,8000]",
                   "buffers": "sized from a measured growth curve (no daughter dropped)", "sizing": sizing,
                   "layout": "FP32 float4 SoA",
                   "timed_from_step": int(s0.step), "parallelism": f"replicas x{world}",
                   "launch": {"graph_steps": K, "tuning": tuning.as_dict(), "autotune_s": round(tune_s, 2)},
                   "l2": "state > L2 (no flush needed)", "tables": "256 chi x 256 r, FP64-built"},
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": 7 * K,  # plan, persistent kernel, event kernel, four compaction kernels per step
        "particles_at_start": {"electrons": int(s0.alive[0]), "positrons": int(s0.alive[1]),
                               "photons": int(s0.alive[2])},
        "particle_steps_timed": {"electrons": d_sp[0], "positrons": d_sp[1], "photons": d_sp[2]},
        "counters": {k: int(v) for k, v in ctr.as_dict().items()},
        "table_build_s": round(t_tables, 2),
    }
    out.update(extras)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return None
    return out


def native_cascade(args):
    """The large cascade (one instance of the batched path): every step of the run timed."""
    import torch
    from paper_2511_08929_gb300 import binding as B
    from paper_2511_08929_gb300 import build as bld
    from paper_2511_08929_gb300 import buffers as Q
    from paper_2511_08929_gb300 import inputs as I
    import dataclasses

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = f"cuda:{local if world > 1 else 0}"
    bld.build()
    wl = I.CASCADE_2E8
    if args.scale != 1.0:
        wl = dataclasses.replace(wl, name=f"{wl.name}_x{args.scale:g}", n_electrons=int(wl.n_electrons * args.scale))
    steps = wl.steps if args.cascade_steps is None else args.cascade_steps
    SEG = min(500, steps)
    ERR_STEPS, ERR_AT = 3, min(1000, steps)
    extras_on = not args.no_extras and rank == 0
    t0 = time.time()
    tables = Q.Tables(1e-4, 1e3, 256, 256)
    torch.cuda.synchronize()
    t_tables = time.time() - t0
    seeds = [wl.seed + 1000 * rank]
    id_offset = np.uint64(rank << 48)
    insts = wl.instances()
    fields = [Q.laser_field(wl.laser())]
    t0 = time.time()
    caps, sizing = growth_capacities(Q, B, tables, wl, insts, fields, seeds, steps + ERR_STEPS + 8, device,
                                     sub=1024, min_sub=4096)
    sizing["seconds"] = round(time.time() - t0, 2)
    bt = Q.Batch(tables, fields, seeds, caps, wl.dt, t0=0.0, step0=0, photon_store_min=wl.photon_store_min,
                 device=device)
    e = bt.buffers()[0][0]
    t0 = time.time()
    done = 0
    for c in range(wl.n_chunks()):
        b = wl.chunk_beam(c)
        if done + len(b["id"]) > wl.n_electrons:
            b = {k: v[:wl.n_electrons - done] for k, v in b.items()}
        e.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"] + id_offset, offset=done)
        done += len(b["id"])
    e.init_tau(seeds[0])
    torch.cuda.synchronize()
    t_load = time.time() - t0
    v, bps, ch = (int(x) for x in (args.tuning or "0,3,16").split(","))
    B.qed_batch_set_tuning(bt.handle, B.QedBatchTuning(v, bps, ch, SEG))
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(SEG)]
    bt.set_kernel_events(kev)
    stream = torch.cuda.current_stream().cuda_stream
    bt.step(0, stream)  # capture and instantiate outside the timed region
    bt.ctr.zero()
    torch.cuda.synchronize()
    stop = threading.Event()
    clock_lines = []
    th = threading.Thread(target=clocks_sampler, args=(stop, clock_lines, local), daemon=True)
    th.start()
    time.sleep(0.5)
    ms, tk, psteps = 0.0, 0.0, 0.0
    d_sp = np.zeros(3)
    tot = {"events": 0, "stored": 0, "rate_steps": 0, "renormalised": 0, "chi_clamped": 0, "below_store": 0}
    growth, extras, timed = [], {}, 0
    s_first = bt.stats(stream)
    while timed < steps:
        n = min(SEG, steps - timed)
        s0 = bt.stats(stream)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        bt.step(n, stream)
        z.record()
        torch.cuda.synchronize()
        ms += a.elapsed_time(z)
        if n == SEG:
            tk += sum(x.elapsed_time(y) for x, y in kev)
        s1 = bt.stats(stream)
        c = bt.ctr.read()
        if c.status != 0:
            raise SystemExit(f"bench: cascade steps ended with status {c.status} ({B.status_string(c.status)}), "
                             f"{c.dropped_capacity} daughters dropped: no valid measurement")
        for k in tot:
            tot[k] += int(getattr(c, k))
        psteps += float(s1.particle_steps - s0.particle_steps)
        d_sp += [float(s1.species_steps[i] - s0.species_steps[i]) for i in range(3)]
        bt.ctr.zero()
        timed += n
        growth.append({"step": int(s1.step), "electrons": int(s1.alive[0]), "positrons": int(s1.alive[1]),
                       "photons": int(s1.alive[2])})
        if extras_on and timed == ERR_AT:  # accuracy mid-cascade (untimed; the batch moves on ERR_STEPS steps)
            alive = int(sum(s1.alive))
            err, cpu = error_leg(bt, wl, fields, seeds, torch, ERR_STEPS, stride=max(16, alive // 200000))
            extras["error"], extras["cpu_baseline"] = err, cpu
            c = bt.ctr.read()
            if c.status != 0:
                raise SystemExit("bench: the error leg's steps overflowed")
            bt.ctr.zero()
    stop.set()
    th.join(timeout=5)
    tmax, psteps_all = ms, psteps
    if dist is not None:
        tmax, psteps_all = reduce_over_ranks(ms, psteps, dist, device)
    value = psteps_all / (tmax / 1e3)
    peak, peak_kind = measured_peaks()
    alg = unit_bytes(d_sp[0] + d_sp[1], d_sp[2], tot["stored"])
    alg_design = design_bytes(d_sp[0] + d_sp[1], d_sp[2], tot["rate_steps"], tot["events"], tot["stored"])
    full = steps // SEG * SEG  # steps whose kernels were event-timed (whole graph launches)
    roof = {"kernel": "batch_step_kernel+batch_event_kernel", "bound": "hbm", "peak": peak, "unit": "GB/s",
            "peak_source": peak_kind, "traffic": None,
            "algorithmic_bytes_per_launch": alg / steps, "design_bytes_per_launch": alg_design / steps}
    if tk > 0:
        achieved = alg * (full / steps) / (tk / 1e3) / 1e9
        roof.update({"achieved": round(achieved, 1), "frac": round(achieved / peak, 4),
                     "frac_design_bytes": round(alg_design * (full / steps) / (tk / 1e3) / 1e9 / peak, 4),
                     "ms_per_launch": round(tk / full, 4), "share_of_step": round(tk / (ms * full / steps), 4)})
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": 0,
        "ms_per_step": tmax / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "electrons_initial": wl.n_electrons, "gamma": wl.gamma,
                   "laser": f"two colliding CP pulses a0={wl.a0:g}, {wl.wavelength_um:g} um, {wl.n_cycles:g} cycles",
                   "photon_store_min_mc2": wl.photon_store_min, "sizing": sizing,
                   "buffers": {"electrons": caps[0][0], "positrons": caps[0][1], "photons": caps[0][2]},
                   "timed": f"all {steps} steps from step 0, graph launches of {SEG} steps",
                   "launch": {"variant": v, "blocks_per_sm": bps, "chunk": ch, "graph_steps": SEG},
                   "parallelism": f"replicas x{world}", "l2": "state > L2 (no flush needed)",
                   "load_s": round(t_load, 1), "tables": "256 chi x 256 r, FP64-built"},
        "roofline": roof,
        "clocks": summarize_clocks(clock_lines),
        "gpu_launches": 7 * steps,
        "growth": growth,
        "particle_steps_timed": {"electrons": d_sp[0], "positrons": d_sp[1], "photons": d_sp[2]},
        "counters": tot,
        "table_build_s": round(t_tables, 2),
    }
    out.update(extras)
    bt.close()
    if dist is not None:
        dist.destroy_process_group()
    return out if rank == 0 else None


class _Workloads:
    """Several head-on workloads as the instances of one batch (the interface growth_capacities reads)."""

    def __init__(self, wls, scale=1.0):
        self.wls = wls
        self.scale = scale
        self.dt = wls[0].dt
        self.photon_store_min = wls[0].photon_store_min

    def instances(self):
        return [{"n": max(1, int(w.n_electrons * self.scale)), "seed": w.seed} for w in self.wls]

    def laser(self, inst):
        return self.wls[self.instances().index(inst)].laser

    def beam(self, k, inst, n=None):
        b = self.wls[k].beam(inst["n"] if n is None else n)
        b["id"] = b["id"] + np.uint64(k << 40)
        return b

    def sample(self, k, inst, m):
        return self.beam(k, inst, m)


def native_helicity(args):
    """The helicity-transfer analogues: both collisions in one batch, every step of the crossing timed."""
    import torch
    from paper_2511_08929_gb300 import binding as B
    from paper_2511_08929_gb300 import build as bld
    from paper_2511_08929_gb300 import buffers as Q
    from paper_2511_08929_gb300 import diagnostics as D
    from paper_2511_08929_gb300 import inputs as I

    torch.cuda.set_device(0)
    device = "cuda:0"
    bld.build()
    tables = Q.Tables(1e-4, 1e3, 256, 256)
    wl = _Workloads([I.HELICITY_LP_X14, I.HELICITY_CP_X15], args.scale)
    insts = wl.instances()
    seeds = [x["seed"] for x in insts]
    fields = [Q.laser_field(w.laser) for w in wl.wls]
    steps = max(w.crossing_steps() for w in wl.wls)
    t0 = time.time()
    caps, sizing = growth_capacities(Q, B, tables, wl, insts, fields, seeds, steps + 8, device, sub=64, min_sub=4096)
    sizing["seconds"] = round(time.time() - t0, 2)
    bt = Q.Batch(tables, fields, seeds, caps, wl.dt, t0=0.0, step0=0, device=device)
    for k, (x, (e, p, g)) in enumerate(zip(insts, bt.buffers())):
        b = z_order(wl.beam(k, x))
        e.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
        e.init_tau(seeds[k])
    v, bps, ch = (int(x) for x in (args.tuning or "0,3,16").split(","))
    SEG = 100
    B.qed_batch_set_tuning(bt.handle, B.QedBatchTuning(v, bps, ch, SEG))
    stream = torch.cuda.current_stream().cuda_stream
    bt.step(0, stream)
    bt.ctr.zero()
    torch.cuda.synchronize()
    stop = threading.Event()
    clock_lines = []
    th = threading.Thread(target=clocks_sampler, args=(stop, clock_lines, 0), daemon=True)
    th.start()
    time.sleep(0.5)
    s0 = bt.stats(stream)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    bt.step(steps, stream)
    z.record()
    torch.cuda.synchronize()
    stop.set()
    th.join(timeout=5)
    ms = a.elapsed_time(z)
    s1 = bt.stats(stream)
    c = bt.ctr.read()
    if c.status != 0:
        raise SystemExit(f"bench: helicity run ended with status {c.status} ({B.status_string(c.status)})")
    psteps = float(s1.particle_steps - s0.particle_steps)
    gev = 1e9 / I.ME_EV
    edges = [i * gev for i in range(0, 11)]
    diag = {}
    for name, (e, p, g) in zip(("x14_lp_photons_xi2", "x15_cp_positrons_longitudinal"), bt.buffers()):
        diag[name] = D.polarization_vs_energy(g if name.startswith("x14") else p, edges)
    diag["energy_unit"] = "m c^2 (bins of 1 GeV)"
    out = {"metric": METRIC, "value": psteps / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": 0,
           "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "helicity_transfer_x14_x15", "instances": [w.name for w in wl.wls],
                      "electrons": [x["n"] for x in insts], "sizing": sizing,
                      "timed": f"all {steps} steps of the crossing, graph launches of {SEG} steps",
                      "launch": {"variant": v, "blocks_per_sm": bps, "chunk": ch}},
           "clocks": summarize_clocks(clock_lines), "gpu_launches": 7 * steps,
           "counters": {k: int(x) for k, x in c.as_dict().items()},
           "particles_at_end": {"electrons": [int(bt.buffers()[k][0].count()) for k in range(2)],
                                "positrons": [int(bt.buffers()[k][1].count()) for k in range(2)],
                                "photons": [int(bt.buffers()[k][2].count()) for k in range(2)]},
           "diagnostics": diag}
    bt.close()
    return out


def headon_leg(args):
    """Config 2 beside the headline: 1e7 electrons (gamma 4000, spin +z) in the CP a0 = 150 pulse through
    the single-buffer FP32 entry points (20 timed steps inside the interaction, buffers sized by the
    growth pass, status 0), and the plain FP64 path on the same state."""
    import copy
    a = copy.copy(args)
    a.workload, a.steps, a.warmup, a.advance, a.electrons = "headon", 20, 3, 620, 10_000_000
    a.no_extras, a.fp64_leg = True, True
    o = native(a)
    v64 = o.get("fp64_plain", {}).get("value")
    return {"workload": o["config"]["workload"], "value": o["value"], "unit": UNIT, "ms_per_step": o["ms_per_step"],
            "roofline": {k: o["roofline"].get(k) for k in ("kernel", "achieved", "frac", "peak")},
            "fp64_plain": o.get("fp64_plain"), "fp32_over_fp64": (o["value"] / v64) if v64 else None,
            "status": o["counters"]["status"], "particles_at_start": o["particles_at_start"],
            "clocks": o["clocks"]}


MLP_WINDOW = 8  # steps per timed window of the learned sampler on the batch's event path


def mlp_event_path(bt, smp, torch, stream, tol=1e-4):
    """The learned sampler inside the batched step (qed_batch_set_mlp) on the timed workload's state:
    four consecutive graph launches of MLP_WINDOW steps each, tables / network / tables / network (the
    alternation cancels the drift of the populations), each captured outside its timed launch."""
    from paper_2511_08929_gb300 import binding as B
    tn = bt.tuning()
    ms = {"tables": 0.0, "network": 0.0}
    ev = {"tables": 0, "network": 0}
    ps = {"tables": 0.0, "network": 0.0}
    fb = 0
    for mode in ("tables", "network", "tables", "network"):
        bt.set_sampler(smp if mode == "network" else None, tol)  # resets the fallback count
        B.qed_batch_set_tuning(bt.handle, B.QedBatchTuning(tn.variant, tn.blocks_per_sm, tn.chunk, MLP_WINDOW))
        bt.step(0, stream)  # capture outside the timed launch
        torch.cuda.synchronize()
        c0, s0 = bt.ctr.read().events, bt.stats(stream).particle_steps
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        bt.step(MLP_WINDOW, stream)
        b.record()
        torch.cuda.synchronize()
        ms[mode] += a.elapsed_time(b)
        ev[mode] += bt.ctr.read().events - c0
        ps[mode] += float(bt.stats(stream).particle_steps - s0)
        if mode == "network":
            fb += bt.sampler_last(0)[1]
    bt.set_sampler(None)
    status = int(bt.ctr.read().status)
    n = 2 * MLP_WINDOW
    return {"steps_per_mode": n, "status": status, "tolerance": tol,
            "ms_per_step_tables": ms["tables"] / n, "ms_per_step_network": ms["network"] / n,
            "events_per_step_tables": ev["tables"] / n, "events_per_step_network": ev["network"] / n,
            "particle_steps_per_s_tables": ps["tables"] / (ms["tables"] / 1e3),
            "particle_steps_per_s_network": ps["network"] / (ms["network"] / 1e3),
            "step_time_ratio_network_over_tables": ms["network"] / ms["tables"],
            "fallback_fraction": fb / max(1, ev["network"]),
            "note": "events counted by the counters (leptons' emissions and photons' pairs); the sampler runs "
                    "on every listed event, pairs with placeholder inputs"}


def mlp_leg(args, tables, torch, bt=None, stream=0):
    """The learned sampler: 3-64-64-64-4 SiLU, BF16 weights and activations with FP32 accumulation on
    tensor cores, trained on table samples at chi in [1e-3, 1e2], evaluated on events with the table
    fallback wherever the network's CDF error (or Stokes error) exceeds 1e-4; the table path beside it;
    with bt, also inside the batched step on its state (mlp_event_path)."""
    from paper_2511_08929_gb300 import mlp as GM
    batch = 4096
    steps = int(math.ceil(args.mlp_train / batch))
    smp = GM.Sampler(GM.init_params(1), max_batch=batch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    losses = smp.train(tables, steps, batch, seed=21, lr=3e-3, lr_final=3e-5)
    e1.record()
    torch.cuda.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3
    lo, hi = math.log(1e-3), math.log(1e2)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)

    def inputs(n):
        chi = torch.exp(lo + (hi - lo) * torch.rand(n, dtype=torch.float64, device="cuda", generator=gen))
        r = torch.rand(n, dtype=torch.float64, device="cuda", generator=gen) * (1 - 2.0 ** -40) + 2.0 ** -41
        s = 2 * torch.rand(n, dtype=torch.float64, device="cuda", generator=gen) - 1
        return chi, r, s

    total, chunk = int(args.mlp_eval), 1 << 24
    done, t_net, n_fb = 0, 0.0, 0
    edges = [0.0, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, float("inf")]
    hist = np.zeros(len(edges) - 1)
    first = None
    while done < total:
        n = min(chunk, total - done)
        chi, r, s = inputs(n)
        if first is None:
            first = (chi, r, s)
        e0.record()
        _, _, nf, err = smp.sample(tables, chi, r, s, tol=1e-4, with_error=True)
        e1.record()
        torch.cuda.synchronize()
        t_net += e0.elapsed_time(e1) / 1e3
        n_fb += int(nf.item())
        hist += np.histogram(err.cpu().numpy(), bins=edges)[0]
        done += n
    chi, r, s = first
    e0.record()
    smp.sample(tables, chi, r, s, table_only=True)
    e1.record()
    torch.cuda.synchronize()
    t_tab = e0.elapsed_time(e1) / 1e3
    smp.sample(tables, chi, r, s, branch_table=True)  # warm-up
    e0.record()
    smp.sample(tables, chi, r, s, branch_table=True)
    e1.record()
    torch.cuda.synchronize()
    t_br = e0.elapsed_time(e1) / 1e3
    net_rate, tab_rate, br_rate = total / t_net, chi.shape[0] / t_tab, chi.shape[0] / t_br
    n_tab = int(chi.shape[0])
    del first, chi, r, s
    torch.cuda.empty_cache()
    event_path = mlp_event_path(bt, smp, torch, stream) if bt is not None else None
    smp.close()
    labels = ["<1e-7", "1e-7..1e-6", "1e-6..1e-5", "1e-5..1e-4", "1e-4..1e-3", ">1e-3"]
    return {"train_samples": steps * batch, "train_steps": steps, "train_s": round(train_s, 2),
            "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-100:].mean()),
            "eval_events": total, "samples_per_s": net_rate, "fallback_fraction": n_fb / total,
            "network_cdf_error_hist": {k: float(v / total) for k, v in zip(labels, hist)},
            "table_path_samples_per_s": tab_rate, "table_path_events": n_tab,
            "table_path": "the checked sampler's own fallback: the exact mixture quantile, regula falsi on the tables' mixture CDF",
            "gain_over_table_path": net_rate / tab_rate,
            "branch_table_samples_per_s": br_rate,
            "branch_table": "the step's sampler: spin branch by W_down(1-s)/(2W_s), one float-float ICDF row",
            "gain_over_branch_table": net_rate / br_rate, "tolerance": 1e-4,
            "parameters": 8836, "weights_bytes_bf16": 2 * (192 + 4096 + 4096 + 256),
            "event_path": event_path}


def _to_fp64(b32, b64, torch):
    """Copy an FP32 buffer's [0, count) into an FP64 buffer (device-side repacking of the qed.h layouts;
    planes of the FP64 buffer: x y z px py pz sx sy sz tau w)."""
    from paper_2511_08929_gb300 import binding as B
    n = b32.count()
    q = b32.q[:, :n]
    P = b64.planes
    P[0:3, :n] = q[0, :, 0:3].T.double()
    if b32.charge == B.QED_PHOTON:
        P[6, :n] = q[0, :, 3].double()
        P[7:9, :n] = q[1, :, 0:2].T.double()
        P[9, :n] = q[1, :, 2:4].contiguous().view(torch.float64).reshape(n)
        P[3:6, :n] = q[2, :, 0:3].T.double()
        P[10, :n] = q[2, :, 3].double()
    else:
        P[3, :n] = q[0, :, 3].double()
        P[4:6, :n] = q[1, :, 0:2].T.double()
        P[6:8, :n] = q[1, :, 2:4].T.double()
        P[8, :n] = q[2, :, 0].double()
        P[10, :n] = q[2, :, 1].double()
        P[9, :n] = q[2, :, 2:4].contiguous().view(torch.float64).reshape(n)
    b64.ids[:n] = b32.ids[:n]
    b64.counts[:] = n


def fp64_leg(bt, wl, fields, seeds, tables, Q, B, torch, stream, steps=3):
    """The plain FP64 path on the batch's current state: every instance through the single-buffer FP64
    entry points (buffers sized for these few steps' growth), particle-steps of the photons, electrons
    and positrons alive at each step's start."""
    step0 = int(bt.stats(stream).step)
    bufs64 = []
    for e, p, g in bt.buffers():
        room = [int(1.1 * b.count()) + 4096 for b in (e, p, g)]
        e64 = Q.ParticleBuffer(room[0], B.QED_FP64, B.QED_ELECTRON, use_begin=True)
        p64 = Q.ParticleBuffer(room[1], B.QED_FP64, B.QED_POSITRON, use_begin=True)
        g64 = Q.ParticleBuffer(room[2], B.QED_FP64, B.QED_PHOTON, photons=True, use_begin=True)
        for a, b in ((e, e64), (p, p64), (g, g64)):
            _to_fp64(a, b, torch)
        bufs64.append((e64, p64, g64, Q.CompactWorkspace(room[2])))
    ctr64 = Q.Counters()
    torch.cuda.synchronize()
    s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    counts = []
    s_.record()
    for k in range(steps):
        counts.append(torch.stack([torch.stack([b.counts[0] for b in x[:3]]).sum() for x in bufs64]).sum())
        s = step0 + k
        for (e64, p64, g64, ws), f, sd in zip(bufs64, fields, seeds):
            d = Q.step_desc(wl.dt, float(s) * wl.dt, s, sd, int(bt.desc.flags), wl.photon_store_min)
            B.qed_snapshot_counts([e64.s, p64.s, g64.s], stream)
            B.qed_pair_step(tables.handle, f, d, g64.s, e64.s, p64.s, ctr64.ptr, stream)
            B.qed_push_step(tables.handle, f, d, e64.s, g64.s, ctr64.ptr, stream)
            B.qed_push_step(tables.handle, f, d, p64.s, g64.s, ctr64.ptr, stream)
            B.qed_compact(g64.s, ws.ptr, ws.bytes, stream)
    e_.record()
    torch.cuda.synchronize()
    ps64 = float(sum(c.item() for c in counts))
    c64 = ctr64.read()
    out = {"value": ps64 / (s_.elapsed_time(e_) / 1e3), "unit": UNIT, "steps": steps,
           "ms_per_step": s_.elapsed_time(e_) / steps, "status": int(c64.status),
           "note": "single-buffer FP64 entry points, instance by instance, from the FP32 batch's state"}
    del bufs64
    torch.cuda.empty_cache()
    return out


def e2e_leg(bt, torch, steps):
    """End to end through the C ABI with host-resident state: every step copies every instance's particle
    planes and ids from pinned host memory to the device, runs one qed_batch_step, and copies the state and
    the counts back."""
    bufs = [b for x in bt.buffers() for b in x]
    n_now = [b.count() for b in bufs]
    host = []
    for b, n in zip(bufs, n_now):
        m = min(b.capacity, int(1.1 * n) + 4096)  # room for these steps' daughters
        hq = torch.empty((3, m, 4), dtype=torch.float32).pin_memory()
        hi = torch.empty(m, dtype=torch.int64).pin_memory()
        hq[:, :n].copy_(b.q[:, :n])
        hi[:n].copy_(b.ids[:n])
        host.append((hq, hi))
    h_counts = torch.empty(len(bufs), dtype=torch.int64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ps_e, bi, bo = 0.0, 0, 0
    for _ in range(steps):
        for (hq, hi), b, nn in zip(host, bufs, n_now):
            for pl in range(3):  # one contiguous copy per float4 plane
                b.q[pl, :nn].copy_(hq[pl, :nn], non_blocking=True)
            b.ids[:nn].copy_(hi[:nn], non_blocking=True)
            bi += 3 * nn * 16 + 8 * nn
        ps_e += sum(n_now)
        bt.step(1)
        h_counts.copy_(torch.stack([b.counts[0] for b in bufs]), non_blocking=True)
        torch.cuda.synchronize()
        n_now = h_counts.tolist()
        for (hq, hi), b, nn in zip(host, bufs, n_now):
            if nn > hq.shape[1]:
                raise RuntimeError("e2e host buffer too small")
            for pl in range(3):
                hq[pl, :nn].copy_(b.q[pl, :nn], non_blocking=True)
            hi[:nn].copy_(b.ids[:nn], non_blocking=True)
            bo += 3 * nn * 16 + 8 * nn
        bo += 8 * len(n_now)
        torch.cuda.synchronize()
    te = time.perf_counter() - t0
    del host
    return {"value": ps_e / te, "unit": UNIT, "h2d_bytes_per_step": bi // steps, "d2h_bytes_per_step": bo // steps,
            "steps": steps,
            "note": "all instances' particle state host-resident, copied in and out through pinned memory every "
                    "step around one qed_batch_step (the steps just before the timed ones)"}


def _oracle_batch_step(O, tb, f, st, E, P, G):
    """One time step of one instance on the oracle, with the begin-snapshot semantics of the batch:
    photons first (pairs appended to E, P), then each lepton species over its particles present at the
    step's start (lepton steps append photons only)."""
    nE, nP = E.n, P.n
    O.photon_step(tb, f, st, G, E, P)
    for L, q, n0 in ((E, -1, nE), (P, 1, nP)):
        n_now = L.n
        L._s.n = n0
        O.lepton_step(tb, f, st, q, L, G)
        L._s.n = n_now


def _oracle_field(O, f):
    return O.field(f.kind, a0=f.a0, n_cycles=f.n_cycles, phase=f.phase, E0=tuple(f.E0), B0=tuple(f.B0), eta0=f.eta0)


def _step_condition(O, f, pre: dict, t: float, dt: float) -> np.ndarray:
    """A lepton step's condition number: max(1, its T-BMT turn |Omega| dt, its field impulse dt (|E| + |B|)
    / |p|), from its state at the step's start (FP64 Boris push, time-centred momentum, standard T-BMT
    vector).  FP32 field rounding, relative to the field's amplitude, reaches the outputs multiplied by
    it: low-energy leptons in strong fields turn their spin by tens of radians in one step."""
    ae = 7.2973525693e-3 / (2.0 * np.pi)
    E, B = O.field_eval_n(_oracle_field(O, f), pre["pos"], t)
    p = pre["mom"]
    h = 0.5 * dt  # the turn's size does not depend on the sign of the charge
    pm = p + h * E
    tv = h * B / np.sqrt(1.0 + (pm * pm).sum(1))[:, None]
    pl = pm + np.cross(pm + np.cross(pm, tv), 2.0 * tv / (1.0 + (tv * tv).sum(1))[:, None])
    pb = 0.5 * (p + pl + h * E)
    g = np.sqrt(1.0 + (pb * pb).sum(1))[:, None]
    b = pb / g
    om = (ae + 1.0 / g) * B - (ae * g / (g + 1.0)) * (b * B).sum(1)[:, None] * b - (ae + 1.0 / (g + 1.0)) * np.cross(b, E)
    pn = np.maximum(np.linalg.norm(p, axis=1), 1e-300)
    imp = dt * (np.linalg.norm(E, axis=1) + np.linalg.norm(B, axis=1)) / pn
    return np.maximum(1.0, np.maximum(np.linalg.norm(om, axis=1) * dt, imp))


def _gpu_rows(buf, idx, torch):
    """rows idx (device int64 tensor) of an FP32 particle buffer, as host FP64 arrays"""
    from paper_2511_08929_gb300 import buffers as Q
    pos, mom, spin, w, tau = Q.unpack32(buf.charge, buf.q[:, idx].cpu().numpy())
    return {"pos": pos, "mom": mom, "spin": spin, "tau": tau, "w": w, "id": buf.ids[idx].cpu().numpy().view(np.uint64).copy()}


def _gpu_find(buf, ids, torch):
    """the rows of an FP32 buffer holding the given ids (host uint64 array): (host arrays of the found rows,
    boolean mask over ids)"""
    n = buf.count()
    have = buf.ids[:n]
    srt, order = torch.sort(have)
    q = torch.from_numpy(np.ascontiguousarray(ids).view(np.int64)).to(have.device)
    pos = torch.searchsorted(srt, q).clamp(max=max(n - 1, 0))
    hit = (srt[pos] == q) if n > 0 else torch.zeros_like(q, dtype=torch.bool)
    rows = order[pos[hit]]
    return _gpu_rows(buf, rows, torch), hit.cpu().numpy()


def _match(g: dict, o: dict):
    """(g rows, o rows) of the ids present in both, in the same order"""
    common, gi, oi = np.intersect1d(g["id"], o["id"], return_indices=True)
    return {k: v[gi] for k, v in g.items()}, {k: v[oi] for k, v in o.items()}


def _errors(g: dict, o: dict, photon: bool):
    """per-particle relative errors of each output: x (floor 1), p or k, s (absolute; photons: P with its
    transverse part's sign free), tau (floor 1)"""
    def rel(a, b, floor):
        return np.linalg.norm(a - b, axis=1) / np.maximum(np.maximum(np.linalg.norm(a, axis=1),
                                                                     np.linalg.norm(b, axis=1)), floor)
    e = {"x": rel(g["pos"], o["pos"], 1.0), ("k" if photon else "p"): rel(g["mom"], o["mom"], 1e-300)}
    sg, so = g["spin"], o["spin"]
    if photon:
        kh = o["mom"] / np.maximum(np.linalg.norm(o["mom"], axis=1, keepdims=True), 1e-300)
        gpar, opar = (sg * kh).sum(1, keepdims=True) * kh, (so * kh).sum(1, keepdims=True) * kh
        flip = ((sg - gpar) * (so - opar)).sum(1) < 0
        sg = np.where(flip[:, None], 2 * gpar - sg, sg)
    e["P" if photon else "s"] = np.linalg.norm(sg - so, axis=1)
    fin = np.isfinite(g["tau"]) & np.isfinite(o["tau"])
    e["tau"] = np.where(fin, np.abs(g["tau"] - o["tau"]) / np.maximum(np.abs(o["tau"]), 1.0), 0.0)
    return e


def error_leg(bt, wl, fields, seeds, torch, steps, stride=16, diverged=1e-3):
    """Each output's error against the FP64 oracle on the benchmark's own state: for `steps` steps, every
    stride-th particle of every instance and species is read before the step, the batch takes the step on
    the GPU, the oracle takes it from the same (FP32, widened) state, and the sampled particles and the
    daughters they made are matched by id.  A particle whose state moved apart by more than `diverged`,
    or a daughter on one side only, is a decision flip.  The oracle's time on this sample is the CPU
    baseline (the oracle as it stands, all host cores)."""
    import oracle as O
    tb = O.tables(1e-4, 1e3, 256, 256)
    acc = {"lepton": {}, "lepton_conditioned": {}, "photon": {}, "daughter": {}}
    n_ps, flips, t_or, ps_or = 0, 0, 0.0, 0
    spec_g, spec_o = [], []
    for _ in range(steps):
        step = int(bt.stats().step)
        pre = []
        for e, p, g in bt.buffers():
            parts = []
            for b in (e, p, g):
                n = b.count()
                parts.append(_gpu_rows(b, torch.arange(0, n, stride, device=b.q.device), torch))
            pre.append(parts)
        bt.step(1)
        torch.cuda.synchronize()
        for k, ((e, p, g), (pe, pp, pg)) in enumerate(zip(bt.buffers(), pre)):
            n0 = [len(x["id"]) for x in (pe, pp, pg)]
            caps = (2 * (n0[0] + n0[2]) + 64, 2 * (n0[1] + n0[2]) + 64, n0[2] + 2 * (n0[0] + n0[1]) + 64)
            E, P, G = (O.Particles.from_arrays(c, d["pos"], d["mom"], d["spin"], d["w"], d["id"], tau=d["tau"])
                       for c, d in zip(caps, (pe, pp, pg)))
            st = O.step_desc(wl.dt, float(step) * wl.dt, step, seeds[k], int(bt.desc.flags), wl.photon_store_min)
            t0 = time.perf_counter()
            _oracle_batch_step(O, tb, _oracle_field(O, fields[k]), st, E, P, G)
            t_or += time.perf_counter() - t0
            ps_or += sum(n0)
            n_ps += sum(n0)
            ov = [x.view() for x in (E, P, G)]
            for (buf, ob, prev, kind) in ((e, ov[0], pe, "lepton"), (p, ov[1], pp, "lepton"), (g, ov[2], pg, "photon")):
                # the sampled particles after the step, then every daughter the oracle made from them
                o_par = {kk: v for kk, v in ob.items() if kk in ("pos", "mom", "spin", "tau", "w", "id")}
                old = np.isin(o_par["id"], prev["id"])
                o_old = {kk: v[old] for kk, v in o_par.items()}
                o_new = {kk: v[~old] for kk, v in o_par.items()}
                g_old, hit_old = _gpu_find(buf, o_old["id"], torch)
                g_new, hit_new = _gpu_find(buf, o_new["id"], torch)
                flips += int((~hit_old).sum()) + int((~hit_new).sum())
                go, oo = _match(g_old, o_old)
                er = _errors(go, oo, kind == "photon")
                bad = np.max(np.stack(list(er.values())), axis=0) > diverged
                flips += int(bad.sum())
                for kk, v in er.items():
                    acc[kind].setdefault(kk, []).append(v[~bad])
                if kind == "lepton":  # the same errors over the step's condition number
                    pm, _ = _match(prev, oo)
                    kap = _step_condition(O, fields[k], pm, float(step) * wl.dt, wl.dt)
                    for kk, v in er.items():
                        acc["lepton_conditioned"].setdefault(kk, []).append((v / kap)[~bad])
                gn, on = _match(g_new, o_new)
                er = _errors(gn, on, kind == "photon")  # the buffer's new particles: daughters of its kind
                bad = np.max(np.stack(list(er.values())), axis=0) > diverged
                flips += int(bad.sum())
                for kk, v in er.items():
                    acc["daughter"].setdefault(f"{'photon' if kind == 'photon' else 'lepton'}_{kk}", []).append(v[~bad])
                if kind == "photon":  # photons emitted this step: the spectrum
                    spec_g.append(np.linalg.norm(gn["mom"][~bad], axis=1))
                    spec_o.append(np.linalg.norm(on["mom"][~bad], axis=1))
            # photons the GPU made from sampled leptons that the oracle did not (flips the other way show
            # in the emitter's state above)

    def q(v):
        v = np.concatenate(v) if v else np.zeros(0)
        if len(v) == 0:
            return None
        return {"n": int(len(v)), "p50": float(np.quantile(v, 0.5)), "p99": float(np.quantile(v, 0.99)),
                "p999": float(np.quantile(v, 0.999)), "max": float(v.max()), "above_1e-5": float((v > 1e-5).mean())}

    out = {"against": "FP64 oracle (oracle/), one step at a time from the GPU's FP32 state",
           "sample": f"every {stride}th particle of every instance and species, {steps} steps",
           "particle_steps": n_ps, "flips": flips, "flip_rate": flips / max(n_ps, 1),
           "diverged_threshold": diverged}
    for kind, d in acc.items():
        out[kind] = {kk: q(v) for kk, v in d.items()}
    sg, so = (np.concatenate(spec_g) if spec_g else np.zeros(0)), (np.concatenate(spec_o) if spec_o else np.zeros(0))
    if len(so):
        rel = np.abs(sg - so) / so
        bins_g = np.floor(64 * np.log10(sg))
        bins_o = np.floor(64 * np.log10(so))
        out["spectrum"] = {"photons": int(len(so)), "rel_err_p99": float(np.quantile(rel, 0.99)),
                           "rel_err_max": float(rel.max()), "bin_64_per_decade_mismatch": int((bins_g != bins_o).sum())}
    cpu = {"value": ps_or / t_or if t_or > 0 else None, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": f"every {stride}th particle of every instance and species of the benchmark's state, "
                     f"{steps} steps ({ps_or} particle-steps, {t_or:.1f} s)"}
    return out, cpu


def reference_arm_batch(args):
    """The oracle, as it stands, on the host cores: the batched workload with every instance reduced
    to a bounded sample of its electrons, advanced to the same window, then W + K timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    from paper_2511_08929_gb300 import inputs as I
    wl = I.BATCHED_96
    insts = wl.instances()
    tb = O.tables(1e-4, 1e3, 256, 256)
    scale = 2e-3
    sample = []
    n_tot = 0
    for k, x in enumerate(insts):
        n = max(1, int(scale * x["n"]))
        b = wl.beam(k, x, n=n)
        L = O.Particles.from_arrays(40 * n + 64, b["pos"], b["mom"], b["spin"], b["w"], b["id"])
        L.init_tau(x["seed"])
        lz = wl.laser(x)
        f = O.field(O.FIELD_LP if lz.kind == "LP" else O.FIELD_CP, a0=lz.a0, n_cycles=lz.n_cycles, phase=lz.phase,
                    eta0=lz.eta0)
        sample.append((L, O.Particles(40 * n + 64), O.Particles(400 * n + 256), f, x["seed"]))
        n_tot += n
    s = 0

    def one():
        nonlocal s
        c = 0
        for E, P, G, f, sd in sample:
            st = O.step_desc(wl.dt, float(s) * wl.dt, s, sd, O.F_FULL, wl.photon_store_min)
            c += E.n + P.n + G.n
            _oracle_batch_step(O, tb, f, st, E, P, G)
        s += 1
        return c
    while s < args.advance:
        one()
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    ps = 0
    for _ in range(args.steps):
        ps += one()
    dt = time.perf_counter() - t0
    v = ps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "instances": len(insts), "sample_electrons": n_tot,
                      "sample": f"{scale:g} of every instance's electrons (at least 1)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": O.num_threads(),
                            "sample": f"{n_tot} electrons over {len(insts)} instances ({scale:g} of each), "
                                      f"steps {args.advance + args.warmup}..{s - 1}"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def extra_legs(args, sim, Q, B, I, wl, tables, device, torch, legs=("fp64", "e2e", "cpu")):
    """e2e through the C ABI with host buffers, the plain FP64 path on the same state, and the oracle
    on a bounded sample of the same state (CPU baseline)."""
    out = {}
    state = sim.state()  # current state (after the timed steps)
    # ---- plain FP64 path on the same state ----
    room = tuple(int(1.1 * b.count()) + 4096 for b in (sim.el, sim.po, sim.ph))
    sim64 = Sim(Q, B, I, wl, B.QED_FP64, tables, sim.n0, sim.seed, room, device)
    sim64.load_state(state)
    sim64.step_index = sim.step_index
    for _ in range(2):
        sim64.step()
    torch.cuda.synchronize()
    K64 = 3
    s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    counts = []
    s_.record()
    for _ in range(K64):
        counts.append(torch.stack([sim64.el.counts[0], sim64.po.counts[0], sim64.ph.counts[0]]).clone())
        sim64.step()
    e_.record()
    torch.cuda.synchronize()
    ps64 = float(sum(c.sum().item() for c in counts))
    v64 = ps64 / (s_.elapsed_time(e_) / 1e3)
    out["fp64_plain"] = {"value": v64, "unit": UNIT, "steps": K64, "ms_per_step": s_.elapsed_time(e_) / K64}
    del sim64
    torch.cuda.empty_cache()
    if "e2e" not in legs:
        return out

    # ---- e2e: host-resident particle state, copied in and out through pinned memory every step ----
    Ke = 3
    host = {}
    for key, buf in (("el", sim.el), ("po", sim.po), ("ph", sim.ph)):
        host[key] = (torch.empty_like(buf.q, device="cpu").pin_memory(), torch.empty_like(buf.ids, device="cpu").pin_memory())
        host[key][0].copy_(buf.q)
        host[key][1].copy_(buf.ids)
    h_counts = torch.empty(3, dtype=torch.int64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ps_e = 0.0
    bi = bo = 0
    for _ in range(Ke):
        n_now = [sim.el.count(), sim.po.count(), sim.ph.count()]
        for (key, buf), nn in zip((("el", sim.el), ("po", sim.po), ("ph", sim.ph)), n_now):
            for pl in range(3):  # one contiguous copy per float4 plane
                buf.q[pl, :nn].copy_(host[key][0][pl, :nn], non_blocking=True)
            buf.ids[:nn].copy_(host[key][1][:nn], non_blocking=True)
            bi += 3 * nn * 16 + 8 * nn
        ps_e += sum(n_now)
        sim.step()
        h_counts.copy_(torch.stack([sim.el.counts[0], sim.po.counts[0], sim.ph.counts[0]]), non_blocking=True)
        torch.cuda.synchronize()
        for (key, buf), nn in zip((("el", sim.el), ("po", sim.po), ("ph", sim.ph)), h_counts.tolist()):
            for pl in range(3):
                host[key][0][pl, :nn].copy_(buf.q[pl, :nn], non_blocking=True)
            host[key][1][:nn].copy_(buf.ids[:nn], non_blocking=True)
            bo += 3 * nn * 16 + 8 * nn
        torch.cuda.synchronize()
    te = time.perf_counter() - t0
    out["e2e"] = {"value": ps_e / te, "unit": UNIT, "h2d_bytes_per_step": bi // Ke, "d2h_bytes_per_step": bo // Ke + 24,
                  "note": "particle state host-resident, copied in and out through pinned memory each step"}

    # ---- CPU baseline: the oracle on a bounded sample of the same state ----
    out["cpu_baseline"] = cpu_baseline(state, wl, sim.step_index, seconds=15.0, n_sample=2_000_000)
    return out


def cpu_baseline(state, wl, step0, seconds=15.0, n_sample=20000, max_steps=40):
    """The oracle on a bounded sample of the same state: n_sample electrons and 4 n_sample photons of
    the current step, at most max_steps steps (so the sample stays inside the interaction) and about
    `seconds` of CPU work."""
    import oracle as O
    tb = O.tables(1e-4, 1e3, 256, 256)
    f = O.field(O.FIELD_CP, a0=wl.laser.a0, n_cycles=wl.laser.n_cycles, phase=wl.laser.phase, eta0=wl.laser.eta0)

    def sample(n):
        sel = {k: v[:n] for k, v in state["el"].items()}
        phs = {k: v[: 4 * n] for k, v in state["ph"].items()}
        L = O.Particles.from_arrays(4 * n, sel["pos"], sel["mom"], sel["spin"], sel["w"], sel["id"], tau=sel["tau"])
        G = O.Particles.from_arrays(8 * n, phs["pos"], phs["mom"], phs["spin"], phs["w"], phs["id"], tau=phs["tau"])
        return L, G, O.Particles(4 * n), O.Particles(4 * n)

    ps, dt, steps = 0, 0.0, 0
    L, G, E, P = sample(n_sample)
    s = step0
    while steps < max_steps and dt < seconds:
        st = O.step_desc(wl.dt, s * wl.dt, s, wl.seed)
        c = L.n + G.n + P.n
        t0 = time.perf_counter()
        O.photon_step(tb, f, st, G, E, P)
        O.lepton_step(tb, f, st, -1, L, G)
        dt += time.perf_counter() - t0
        ps += c
        s += 1
        steps += 1
    return {"value": ps / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n_sample} electrons + {min(len(state['ph']['id']), 4 * n_sample)} photons of the benchmark's "
                      f"state at step {step0}, {steps} steps, {dt:.1f} s"}


def reference_arm(args):
    """The oracle, as it stands, on the host cores: same metric and config, each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    from paper_2511_08929_gb300 import inputs as I
    wl = I.HEADON_CP_LARGE
    n = 20000
    beam = I.lepton_beam(n, wl.gamma, direction=(0.0, 0.0, -1.0), z_range=(2 * math.pi, 22 * math.pi), spin="fixed",
                         spin_dir=(0.0, 0.0, 1.0), seed=wl.seed)
    tb = O.tables(1e-4, 1e3, 256, 256)
    L = O.Particles.from_arrays(4 * n, beam["pos"], beam["mom"], beam["spin"], beam["w"], beam["id"])
    L.init_tau(wl.seed)
    G, E, P = O.Particles(40 * n), O.Particles(4 * n), O.Particles(4 * n)
    f = O.field(O.FIELD_CP, a0=wl.laser.a0, n_cycles=wl.laser.n_cycles, phase=wl.laser.phase, eta0=wl.laser.eta0)
    s = 0
    def one():
        nonlocal s
        st = O.step_desc(wl.dt, s * wl.dt, s, wl.seed)
        c = L.n + G.n + P.n
        O.photon_step(tb, f, st, G, L, P)
        O.lepton_step(tb, f, st, -1, L, G)
        s += 1
        return c
    while s < args.advance:  # reach the interaction with the small sample (untimed)
        one()
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    ps = 0
    for _ in range(args.steps):
        ps += one()
    dt = time.perf_counter() - t0
    v = ps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "sample_electrons": n},
           "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": O.num_threads(),
                            "sample": f"{n} electrons of the same beam, {args.steps} steps"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main() or 0)
