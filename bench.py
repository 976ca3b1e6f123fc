"""Throughput of the spin/polarization-resolved QED step on GB300.

Workload (default): 1e7 electrons, gamma 4000, spin +z, head-on with a circularly polarized plane wave
(a0 = 150 per component, 0.8 um, 20-cycle sin^2 envelope), NLC + polarization-resolved NBW, daughters
appended to buffers of 4x the initial count, dt = lambda/(100 c), FP32 path (FP64 optical depth).
The beam is advanced (untimed) to the middle of the interaction, then W warm-up steps and K timed
steps run.  One step = snapshot of the counts, the photon (pair) step, the electron and positron
(emission) steps and the compaction of converted photons; its particle-steps are the photons,
electrons and positrons alive at the step's start.  The particle state (~2.4 GB) is far larger than
L2, so no flush is needed between steps.

Multi-GPU (torchrun): every rank runs an independent replica of the workload with its own seed
(particles never interact across ranks; there is no data-path collective): weak scaling.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
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

METRIC = "QED particle-steps/s (FP32 path, head-on CP a0=150 collision, NLC + NBW)"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--electrons", type=int, default=10_000_000)
    ap.add_argument("--advance", type=int, default=620, help="untimed steps before warm-up (reach the pulse)")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, e2e and CPU-baseline legs")
    return ap.parse_args()


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

    def __init__(self, Q, B, I, wl, layout, tables, n, seed, cap_factor, device):
        import torch
        self.Q, self.B, self.torch = Q, B, torch
        self.wl = wl
        self.tables = tables
        self.field = Q.laser_field(wl.laser)
        cap = int(cap_factor * n)
        self.el = Q.ParticleBuffer(cap, layout, B.QED_ELECTRON, device=device, use_begin=True)
        self.po = Q.ParticleBuffer(cap, layout, B.QED_POSITRON, device=device, use_begin=True)
        self.ph = Q.ParticleBuffer(cap, layout, B.QED_PHOTON, device=device, photons=True, use_begin=True)
        self.ws = Q.CompactWorkspace(cap, device=device)
        self.ctr = Q.Counters(device=device)
        self.seed = seed
        self.n0 = n
        self.step_index = 0
        self.stream = torch.cuda.current_stream().cuda_stream

    def load_beam(self, beam):
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
        return reference_arm(args)
    out = native(args)
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
    sim = Sim(Q, B, I, wl, B.QED_FP32, tables, n, seed, wl.capacity_factor, device)
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
    h = hist.cpu().numpy().astype(np.float64)
    psteps = float(h.sum())
    n_el, n_po, n_ph = h[:, 0].sum(), h[:, 1].sum(), h[:, 2].sum()
    tmax = ms
    psteps_all = psteps
    if dist is not None:
        t = torch.tensor([ms], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax = float(t.item())
        p = torch.tensor([psteps], device=device, dtype=torch.float64)
        dist.all_reduce(p)
        psteps_all = float(p.item())
    value = psteps_all / (tmax / 1e3)

    # roofline of the dominant kernel: algorithmic bytes per launch / its event-timed duration
    # electron step: 88 B per lepton-step (read x, p, s, tau 44 B; write x, p, s, tau 44 B)
    #                + 8 B id per emission + 52 B per stored photon (x, k, P 36 + tau 8 + id 8)
    # photon step:   76 B per photon-step (read x, k, P, tau 44 B; write x, P, tau 32 B)
    #                + 8 B id per conversion + 104 B per stored pair
    peak, peak_kind = measured_peaks()
    push_bytes = 88.0 * n_el + 60.0 * (ctr.events)  # events of all species counted together (upper bound)
    pair_bytes = 76.0 * n_ph
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
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": tmax / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "electrons_per_gpu": n, "gamma": wl.gamma, "a0": wl.laser.a0,
                   "laser": "CP 0.8um 20 cycles", "buffers": "4x initial per species", "layout": "FP32 float4 SoA",
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


def extra_legs(args, sim, Q, B, I, wl, tables, device, torch):
    """e2e through the C ABI with host buffers, the plain FP64 path on the same state, and the oracle
    on a bounded sample of the same state (CPU baseline)."""
    out = {}
    state = sim.state()  # current state (after the timed steps)
    # ---- plain FP64 path on the same state ----
    sim64 = Sim(Q, B, I, wl, B.QED_FP64, tables, sim.n0, sim.seed, wl.capacity_factor, device)
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
            buf.q[:, :nn].copy_(host[key][0][:, :nn], non_blocking=True)
            buf.ids[:nn].copy_(host[key][1][:nn], non_blocking=True)
            bi += 3 * nn * 16 + 8 * nn
        ps_e += sum(n_now)
        sim.step()
        h_counts.copy_(torch.stack([sim.el.counts[0], sim.po.counts[0], sim.ph.counts[0]]), non_blocking=True)
        torch.cuda.synchronize()
        for (key, buf), nn in zip((("el", sim.el), ("po", sim.po), ("ph", sim.ph)), h_counts.tolist()):
            host[key][0][:, :nn].copy_(buf.q[:, :nn], non_blocking=True)
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
