"""Device memory for the C ABI: particle buffers as PyTorch CUDA tensors, the table handle, and the
field / step descriptors.  PyTorch only allocates memory and provides streams here; every step of the
method runs in libqedgb's kernels (see binding.py)."""
from __future__ import annotations


import numpy as np
import torch

from . import binding as B

PLANES64 = ("x", "y", "z", "px", "py", "pz", "sx", "sy", "sz", "tau", "w")


def pack32(charge: int, pos, mom, spin, w, tau) -> np.ndarray:
    """(3, n, 4) float32 planes of the FP32 layout (qed.h): leptons q0 = (x, y, z, px),
    q1 = (py, pz, sx, sy), q2 = (sz, w, tau_lo, tau_hi); photons q0 = (x, y, z, sx), q1 = (sy, sz, tau_lo,
    tau_hi), q2 = (px, py, pz, w); tau as the two 32-bit words of its FP64 bit pattern."""
    n = len(w)
    host = np.zeros((3, n, 4), dtype=np.float32)
    tw = np.asarray(tau, dtype=np.float64).view(np.uint32).reshape(n, 2).view(np.float32)
    host[0, :, 0:3] = pos
    if charge == B.QED_PHOTON:
        host[0, :, 3] = spin[:, 0]
        host[1, :, 0:2] = spin[:, 1:3]
        host[1, :, 2:4] = tw
        host[2, :, 0:3] = mom
        host[2, :, 3] = w
    else:
        host[0, :, 3] = mom[:, 0]
        host[1, :, 0:2] = mom[:, 1:3]
        host[1, :, 2:4] = spin[:, 0:2]
        host[2, :, 0] = spin[:, 2]
        host[2, :, 1] = w
        host[2, :, 2:4] = tw
    return host


def unpack32(charge: int, h: np.ndarray):
    """(pos, mom, spin, w, tau) as FP64 arrays from (3, n, 4) planes of the FP32 layout"""
    n = h.shape[1]
    pos = h[0, :, 0:3].astype(np.float64)
    if charge == B.QED_PHOTON:
        spin = np.column_stack([h[0, :, 3], h[1, :, 0], h[1, :, 1]]).astype(np.float64)
        mom = h[2, :, 0:3].astype(np.float64)
        w = h[2, :, 3].astype(np.float64)
        tw = h[1, :, 2:4]
    else:
        mom = np.column_stack([h[0, :, 3], h[1, :, 0], h[1, :, 1]]).astype(np.float64)
        spin = np.column_stack([h[1, :, 2], h[1, :, 3], h[2, :, 0]]).astype(np.float64)
        w = h[2, :, 1].astype(np.float64)
        tw = h[2, :, 2:4]
    tau = np.ascontiguousarray(tw).view(np.uint32).reshape(n, 2).copy().view(np.float64).reshape(n)
    return pos, mom, spin, w, tau


class ParticleBuffer:
    """One species in the layout qed.h describes: QED_FP64 (eleven double planes) or QED_FP32 (three
    float4 planes; see pack32)."""

    def __init__(self, capacity: int, layout: int, charge: int, device="cuda", photons: bool = False,
                 use_begin: bool = False):
        self.capacity = int(capacity)
        self.layout = layout
        self.charge = charge
        cap = max(self.capacity, 1)
        dev = torch.device(device)
        self.device = dev
        self.s = B.QedParticles()
        self.s.layout = layout
        self.s.charge = charge
        self.s.capacity = self.capacity
        if layout == B.QED_FP64:
            self.planes = torch.zeros((11, cap), dtype=torch.float64, device=dev)
            for i, n in enumerate(PLANES64):
                setattr(self.s, n, self.planes[i].data_ptr())
        else:
            self.q = torch.zeros((3, cap, 4), dtype=torch.float32, device=dev)
            for i in range(3):
                setattr(self.s, f"q{i}", self.q[i].data_ptr())
        self.ids = torch.zeros(cap, dtype=torch.int64, device=dev)
        self.s.id = self.ids.data_ptr()
        self.counts = torch.zeros(2, dtype=torch.int64, device=dev)  # [count, begin]
        self.s.count = self.counts.data_ptr()
        # begin is opt-in: a caller that sets it must refresh it each step (qed_snapshot_counts)
        self.s.begin = self.counts[1:].data_ptr() if use_begin else None
        if photons:
            self.dead = torch.zeros(cap, dtype=torch.int64, device=dev)
            self.n_dead = torch.zeros(1, dtype=torch.int64, device=dev)
            self.s.dead = self.dead.data_ptr()
            self.s.n_dead = self.n_dead.data_ptr()

    # ---- host <-> device marshalling -----------------------------------------------------
    def load(self, pos, mom, spin, w, ids, tau=None, offset=0):
        """Copy host arrays (n, 3), (n, 3), (n, 3), (n,), (n,) [and tau (n,)] into [offset, offset + n) and
        set the count to offset + n (loading a beam in chunks: offset = particles already loaded)."""
        n = len(ids)
        if offset < 0 or offset + n > self.capacity:
            raise ValueError("capacity")
        pos, mom, spin = (np.asarray(a, dtype=np.float64).reshape(n, 3) for a in (pos, mom, spin))
        w = np.asarray(w, dtype=np.float64).reshape(n)
        tau = np.zeros(n) if tau is None else np.asarray(tau, dtype=np.float64).reshape(n)
        if self.layout == B.QED_FP64:
            host = np.empty((11, n))
            host[0:3] = pos.T
            host[3:6] = mom.T
            host[6:9] = spin.T
            host[9] = tau
            host[10] = w
            self.planes[:, offset:offset + n].copy_(torch.from_numpy(host))
        else:
            self.q[:, offset:offset + n].copy_(torch.from_numpy(pack32(self.charge, pos, mom, spin, w, tau)))
        self.ids[offset:offset + n].copy_(torch.from_numpy(np.asarray(ids, dtype=np.uint64).view(np.int64)))
        self.counts.copy_(torch.tensor([offset + n, offset + n], dtype=torch.int64))
        if hasattr(self, "n_dead"):
            self.n_dead.zero_()

    def count(self) -> int:
        return int(self.counts[0].item())

    def read(self, limit=None) -> dict:
        """Host copy of [0, count) (or of its first `limit` particles) as FP64 arrays (pos, mom, spin,
        tau, w, id)."""
        n = self.count()
        if limit is not None:
            n = min(n, int(limit))
        if self.layout == B.QED_FP64:
            h = self.planes[:, :n].cpu().numpy()
            pos, mom, spin, tau, w = h[0:3].T.copy(), h[3:6].T.copy(), h[6:9].T.copy(), h[9].copy(), h[10].copy()
        else:
            pos, mom, spin, w, tau = unpack32(self.charge, self.q[:, :n].cpu().numpy())
        ids = self.ids[:n].cpu().numpy().view(np.uint64).copy()
        return {"pos": pos, "mom": mom, "spin": spin, "tau": tau, "w": w, "id": ids}

    def init_tau(self, seed: int, begin: int = 0, stream: int = 0):
        B.qed_init_tau(self.s, seed, begin, stream)

    def bytes_per_particle(self) -> int:
        return (88 if self.layout == B.QED_FP64 else 48) + 8


class Tables:
    """Owner of a qed_tables_t handle."""

    def __init__(self, chi_min=1e-4, chi_max=1e3, n_chi=256, n_r=256, y_lo=-20.0, y_hi=20.0, stream: int = 0):
        self.desc = B.QedTableDesc(chi_min, chi_max, n_chi, n_r, y_lo, y_hi)
        self.handle = B.qed_tables_build(self.desc, stream)

    def export(self):
        return B.qed_tables_export(self.handle, self.desc)

    def close(self):
        if self.handle:
            B.qed_tables_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def field(kind=B.QED_FIELD_LP, a0=0.0, n_cycles=10.0, phase=0.0, E0=(0, 0, 0), B0=(0, 0, 0),
          eta0=3.0329e-6) -> B.QedField:
    f = B.QedField()
    f.kind = kind
    f.a0 = a0
    f.n_cycles = n_cycles
    f.phase = phase
    for i in range(3):
        f.E0[i] = E0[i]
        f.B0[i] = B0[i]
    f.eta0 = eta0
    return f


def step_desc(dt, t, step, seed, flags=None, photon_store_min=0.0, chi_floor=0.0) -> B.QedStepDesc:
    s = B.QedStepDesc()
    s.dt = dt
    s.t = t
    s.step = step
    s.seed = seed
    s.flags = B.QED_F_FULL if flags is None else flags
    s.photon_store_min = photon_store_min
    s.chi_floor = chi_floor
    return s


class Counters:
    """Device-resident qed_counters."""

    def __init__(self, device="cuda"):
        self.t = torch.zeros(16, dtype=torch.int64, device=device)  # 128 bytes >= sizeof(qed_counters)
        self.ptr = self.t.data_ptr()

    def zero(self):
        self.t.zero_()

    def read(self, stream: int = 0) -> B.QedCounters:
        return B.qed_counters_read(self.ptr, stream)


class CompactWorkspace:
    def __init__(self, capacity: int, device="cuda"):
        self.bytes = B.qed_compact_workspace_bytes(capacity)
        self.t = torch.zeros((self.bytes + 15) // 16 * 2, dtype=torch.int64, device=device)
        self.ptr = self.t.data_ptr()


class Batch:
    """A batch of independent collisions (qed_batch_*): per instance an FP32 electron, positron and
    photon buffer, a laser and a Philox seed; all instances advance together in one persistent launch
    per time step."""

    def __init__(self, tables: "Tables", fields, seeds, capacities, dt, t0=0.0, step0=0, flags=None,
                 photon_store_min=0.0, chi_floor=0.0, device="cuda"):
        """fields: QedField per instance; seeds: Philox seed per instance; capacities: (electrons,
        positrons, photons) capacity per instance."""
        self.device = torch.device(device)
        self.el, self.po, self.ph = [], [], []
        insts = []
        for f, sd, (ce, cp, cg) in zip(fields, seeds, capacities):
            e = ParticleBuffer(ce, B.QED_FP32, B.QED_ELECTRON, device=device)
            p = ParticleBuffer(cp, B.QED_FP32, B.QED_POSITRON, device=device)
            g = ParticleBuffer(cg, B.QED_FP32, B.QED_PHOTON, device=device, photons=True)
            self.el.append(e)
            self.po.append(p)
            self.ph.append(g)
            inst = B.QedInstance()
            inst.field = f
            inst.seed = int(sd)
            inst.electrons, inst.positrons, inst.photons = e.s, p.s, g.s
            insts.append(inst)
        self.desc = B.QedBatchDesc()
        self.desc.dt, self.desc.t0, self.desc.step0 = dt, t0, step0
        self.desc.flags = B.QED_F_FULL if flags is None else flags
        self.desc.photon_store_min, self.desc.chi_floor = photon_store_min, chi_floor
        self.ctr = Counters(device)
        self.tables = tables
        self.handle = B.qed_batch_create(tables.handle, insts, self.desc, self.ctr.ptr)

    def __len__(self):
        return len(self.el)

    def step(self, n_steps: int = 1, stream: int = 0):
        B.qed_batch_step(self.handle, n_steps, stream)

    def tune(self, steps_per_candidate: int = 2, cache_path=None, stream: int = 0):
        return B.qed_batch_tune(self.handle, steps_per_candidate, cache_path, stream)

    def set_tuning(self, variant=0, blocks_per_sm=0, chunk=4, graph_steps=8):
        t = B.QedBatchTuning(variant, blocks_per_sm, chunk, graph_steps)
        B.qed_batch_set_tuning(self.handle, t)

    def tuning(self):
        return B.qed_batch_get_tuning(self.handle)

    def set_kernel_events(self, events):
        """events: list of (start, end) torch.cuda.Event pairs (timing enabled) recorded around the
        persistent kernel of successive steps (see qed_batch_set_kernel_events)."""
        for pair in events:  # torch creates the CUDA event at its first record
            for e in pair:
                if not e.cuda_event:
                    e.record()
        torch.cuda.synchronize(self.device)
        flat = [e.cuda_event for pair in events for e in pair]
        B.qed_batch_set_kernel_events(self.handle, flat, len(events))

    def stats(self, stream: int = 0):
        return B.qed_batch_stats_read(self.handle, stream)

    def set_sampler(self, sampler=None, tol: float = 1e-4):
        """Draw every emission's energy fraction with the learned sampler (an mlp.Sampler, kept alive by
        this batch while it is set), checked at tol with the tables as fallback; None restores the
        tables."""
        B.qed_batch_set_mlp(self.handle, sampler.handle if sampler is not None else None, tol)
        self._sampler = sampler

    def sampler_last(self, n_max: int):
        """The last step's sampler inputs and outputs (see binding.qed_batch_mlp_last)."""
        return B.qed_batch_mlp_last(self.handle, n_max)

    def buffers(self):
        return [(self.el[k], self.po[k], self.ph[k]) for k in range(len(self))]

    def close(self):
        if getattr(self, "handle", None):
            B.qed_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def laser_field(laser, kind_map=None) -> B.QedField:
    """qed_field of an inputs.Laser."""
    kinds = {"LP": B.QED_FIELD_LP, "CP": B.QED_FIELD_CP, "CP_COUNTER": B.QED_FIELD_CP_COUNTER}
    return field(kinds[laser.kind], a0=laser.a0, n_cycles=laser.n_cycles, phase=laser.phase, eta0=laser.eta0)


def sizeof_counters() -> int:
    import ctypes
    return ctypes.sizeof(B.QedCounters)


assert sizeof_counters() <= 128
