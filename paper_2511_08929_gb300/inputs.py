"""Seeded synthetic inputs: particle beams, laser parameters and the named workloads.

This module holds no arithmetic of the QED method: it only draws initial particle
states (positions, momenta, spins, polarizations, weights, ids) with numpy's
seeded generator and records workload parameters.  Both the CUDA path and the
CPU oracle start from these arrays.  The random numbers the method itself draws
(optical depths, energy fractions, collapses, daughter ids) are not made here:
each side derives them from its own Philox4x32-10 keyed by (id, step).

Units: time 1/omega, length c/omega, momentum m c, fields m c omega / e.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ME_EV = 510998.95  # electron rest energy, eV
HC_EV_NM = 1239.841984  # h c, eV nm


def eta0_for_wavelength(wavelength_um: float) -> float:
    """hbar omega / (m c^2) of a laser of the given wavelength."""
    return HC_EV_NM / (wavelength_um * 1000.0) / ME_EV


def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def lepton_beam(n: int, gamma: float, *, rel_spread: float = 0.0, ang_sigma: float = 0.0,
                direction=(0.0, 0.0, -1.0), z_range=(0.0, 0.0), transverse=0.0, spin="random",
                spin_dir=(0.0, 0.0, 1.0), degree: float = 1.0, seed: int = 0, id_offset: int = 0,
                weight: float = 1.0) -> dict:
    """A beam of n leptons with mean Lorentz factor `gamma`.

    spin: "random"  -- independent uniformly distributed unit vectors (unpolarized ensemble)
          "fixed"   -- all along spin_dir
          "degree"  -- +-spin_dir with P(+) = (1 + degree)/2 (partially polarized, pure states)
          "zero"    -- s = 0 (mixed, unpolarized macro-particles)
    """
    rng = np.random.default_rng(seed)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    g = gamma * (1.0 + rel_spread * rng.normal(size=n)) if rel_spread > 0 else np.full(n, float(gamma))
    g = np.maximum(g, 1.0 + 1e-9)
    pmag = np.sqrt(g * g - 1.0)
    # two unit vectors orthogonal to d
    a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(d, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    th1 = ang_sigma * rng.normal(size=n) if ang_sigma > 0 else np.zeros(n)
    th2 = ang_sigma * rng.normal(size=n) if ang_sigma > 0 else np.zeros(n)
    dirs = d[None, :] + th1[:, None] * e1[None, :] + th2[:, None] * e2[None, :]
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    mom = dirs * pmag[:, None]
    pos = np.zeros((n, 3))
    pos[:, 2] = rng.uniform(z_range[0], z_range[1], size=n) if z_range[1] > z_range[0] else z_range[0]
    if transverse > 0:
        pos[:, 0] = rng.uniform(-transverse, transverse, size=n)
        pos[:, 1] = rng.uniform(-transverse, transverse, size=n)
    sd = np.asarray(spin_dir, dtype=np.float64)
    sd = sd / np.linalg.norm(sd)
    if spin == "random":
        s = _unit_vectors(rng, n)
    elif spin == "fixed":
        s = np.tile(sd, (n, 1))
    elif spin == "degree":
        sign = np.where(rng.uniform(size=n) < 0.5 * (1.0 + degree), 1.0, -1.0)
        s = sign[:, None] * sd[None, :]
    elif spin == "zero":
        s = np.zeros((n, 3))
    else:
        raise ValueError(spin)
    ids = np.arange(id_offset, id_offset + n, dtype=np.uint64)
    return {"pos": pos, "mom": mom, "spin": s, "w": np.full(n, float(weight)), "id": ids}


def photon_beam(n: int, energy: float, *, direction=(1.0, 0.0, 0.0), P=(0.0, 1.0, 0.0), seed: int = 0,
                id_offset: int = 0, weight: float = 1.0, P_list=None) -> dict:
    """n photons of energy `energy` (units of m c^2) along `direction`, polarization vector P
    (or P_list, cycled over the photons)."""
    rng = np.random.default_rng(seed)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    mom = np.tile(d * energy, (n, 1))
    pos = np.zeros((n, 3))
    pos[:, 0] = rng.uniform(-1.0, 1.0, size=n) * 0.0
    if P_list is not None:
        Ps = np.asarray(P_list, dtype=np.float64)
        pol = Ps[np.arange(n) % len(Ps)]
    else:
        pol = np.tile(np.asarray(P, dtype=np.float64), (n, 1))
    ids = np.arange(id_offset, id_offset + n, dtype=np.uint64)
    return {"pos": pos, "mom": mom, "spin": pol, "w": np.full(n, float(weight)), "id": ids}


def random_states(n: int, *, seed: int, gamma_range=(50.0, 5000.0), field_region=(-30.0, 30.0)) -> dict:
    """Generic lepton states scattered over a collision region (used to exercise every branch in
    one step): log-uniform gamma, random directions near -z, random pure/mixed spins."""
    rng = np.random.default_rng(seed)
    g = np.exp(rng.uniform(math.log(gamma_range[0]), math.log(gamma_range[1]), size=n))
    pm = np.sqrt(g * g - 1.0)
    d = np.column_stack([rng.normal(0, 0.05, n), rng.normal(0, 0.05, n), -np.ones(n)])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    mom = d * pm[:, None]
    pos = np.column_stack([rng.uniform(-5, 5, n), rng.uniform(-5, 5, n), rng.uniform(*field_region, n)])
    s = _unit_vectors(rng, n) * np.where(rng.uniform(size=n) < 0.7, 1.0, rng.uniform(size=n))[:, None]
    return {"pos": pos, "mom": mom, "spin": s, "w": rng.uniform(0.5, 2.0, n), "id": np.arange(n, dtype=np.uint64) * 7919 + 13}


# ----------------------------------------------------------------------------------------------
# Named workloads (synthetic stand-ins for the paper's laser-beam collisions)
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Laser:
    kind: str  # "LP", "CP", "CP_COUNTER", "CONST"
    a0: float
    wavelength_um: float
    n_cycles: float
    phase: float = 0.0

    @property
    def eta0(self) -> float:
        return eta0_for_wavelength(self.wavelength_um)


@dataclasses.dataclass
class Workload:
    name: str
    n_electrons: int
    gamma: float
    laser: Laser
    steps: int
    dt: float = 2.0 * math.pi / 100.0  # lambda / (100 c)
    rel_spread: float = 0.0
    ang_sigma: float = 0.0
    spin: str = "random"
    spin_dir: tuple = (0.0, 0.0, 1.0)
    pairs: bool = False
    capacity_factor: float = 4.0
    n_chi: int = 256
    n_r: int = 256
    seed: int = 1
    photon_store_min: float = 0.0
    z_cycles: float = 10.0  # beam length in wavelengths (electrons at z in [lambda, (1 + z_cycles) lambda])

    def beam(self, n=None, seed=None):
        n = self.n_electrons if n is None else n
        lam = 2.0 * math.pi  # wavelength in c/omega
        return lepton_beam(n, self.gamma, rel_spread=self.rel_spread, ang_sigma=self.ang_sigma,
                           direction=(0.0, 0.0, -1.0), z_range=(lam, (1.0 + self.z_cycles) * lam), spin=self.spin,
                           spin_dir=self.spin_dir, seed=self.seed if seed is None else seed)

    def crossing_steps(self) -> int:
        """Steps for the whole beam to cross the whole pulse (closing speed 2c) and leave it."""
        return int(math.ceil((self.laser.n_cycles + self.z_cycles + 1.0) * 2.0 * math.pi / 2.0 / self.dt)) + 20


# 1e4 electrons, gamma 2000 (1 % spread, 1 mrad), random unit spins, LP a0=50, 0.8 um, 10 cycles,
# 2000 steps, emission only, tables 256 x 256, seed 1.
HEADON_LP_SMALL = Workload("headon_lp_a50_g2000_n1e4", 10_000, 2000.0, Laser("LP", 50.0, 0.8, 10.0), 2000,
                           rel_spread=0.01, ang_sigma=1e-3, spin="random", seed=1)
# 1e7 electrons, gamma 4000, s = +z, CP a0=150, 20 cycles, 4000 steps, NLC + NBW, buffers 4x.
HEADON_CP_LARGE = Workload("headon_cp_a150_g4000_n1e7", 10_000_000, 4000.0, Laser("CP", 150.0, 0.8, 20.0), 4000,
                           spin="fixed", spin_dir=(0.0, 0.0, 1.0), pairs=True, capacity_factor=4.0, seed=2)


# Plane-wave analogues of the helicity-transfer benchmarks of Sec. 8.6.3 and 8.6.4 (focused pulses there):
# 10 GeV electrons (6 % spread), fully longitudinally polarized with helicity +1 (spin along the momentum,
# -z), a 2-wavelength bunch, against
#   X14: a linearly polarized pulse a0 = 50, 1 um, 12 cycles: circularly polarized photons;
#   X15: a circularly polarized pulse a0 = 100, 1 um, 5 cycles: longitudinally polarized positrons.
HELICITY_LP_X14 = Workload("helicity_lp_a50_10GeV", 1_000_000, 10e9 / ME_EV, Laser("LP", 50.0, 1.0, 12.0), 0,
                           rel_spread=0.06, spin="fixed", spin_dir=(0.0, 0.0, -1.0), pairs=True, seed=14,
                           z_cycles=2.0)
HELICITY_CP_X15 = Workload("helicity_cp_a100_10GeV", 1_000_000, 10e9 / ME_EV, Laser("CP", 100.0, 1.0, 5.0), 0,
                           rel_spread=0.06, spin="fixed", spin_dir=(0.0, 0.0, -1.0), pairs=True, seed=15,
                           z_cycles=2.0)


@dataclasses.dataclass
class BatchWorkload:
    """Many independent collisions stepped together (see batched_instances for the draws)."""
    name: str
    n_inst: int
    n_min: float
    n_max: float
    wavelength_um: float = 0.8
    n_cycles: float = 10.0
    steps: int = 2000
    dt: float = 2.0 * math.pi / 100.0
    capacity_factor: float = 4.0
    n_chi: int = 256
    n_r: int = 256
    seed: int = 3
    photon_store_min: float = 0.0

    def instances(self):
        return batched_instances(self.n_inst, self.seed, self.n_min, self.n_max)

    def laser(self, inst) -> Laser:
        return Laser(inst["kind"], inst["a0"], self.wavelength_um, self.n_cycles)

    def beam(self, k: int, inst, n=None) -> dict:
        """Electrons of instance k: counter-propagating along -z, z0 ~ U[lambda, 11 lambda], spins +-n_k
        with P(+) = (1 + d_k)/2; ids k 2^40 + i."""
        lam = 2.0 * math.pi
        return lepton_beam(inst["n"] if n is None else n, inst["gamma"], direction=(0.0, 0.0, -1.0),
                           z_range=(lam, 11.0 * lam), spin="degree", spin_dir=inst["spin_dir"],
                           degree=inst["degree"], seed=inst["seed"], id_offset=k << 40)


def batched_instances(n_inst: int = 96, seed: int = 3, n_min: float = 1e3, n_max: float = 2e6):
    """Independent collisions of uneven sizes: N log-uniform in [n_min, n_max], a0 ~ U[10, 300],
    gamma ~ U[500, 8000], spins +-n_i with P(+) = (1 + d_i)/2, d_i ~ U[0, 1]; LP and CP alternate."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        a0 = float(rng.uniform(10.0, 300.0))
        g = float(rng.uniform(500.0, 8000.0))
        nd = rng.normal(size=3)
        nd /= np.linalg.norm(nd)
        deg = float(rng.uniform(0.0, 1.0))
        out.append({"n": n, "a0": a0, "gamma": g, "spin_dir": tuple(nd), "degree": deg,
                    "kind": "LP" if i % 2 == 0 else "CP", "seed": int(rng.integers(1 << 31))})
    return out


# 96 collisions, N log-uniform in [1e3, 2e6] (about 2.5e7 electrons in all), a0 ~ U[10, 300],
# gamma ~ U[500, 8000], partially polarized spins, LP / CP alternating, 0.8 um, 10 cycles, 2000 steps,
# NLC + NBW, buffers 4x per species.
BATCHED_96 = BatchWorkload("batched96_n1e3-2e6_a10-300_g500-8000", 96, 1e3, 2e6)


@dataclasses.dataclass
class CascadeWorkload:
    """Electrons seeded where two circularly polarized pulses collide head on (the plane-wave stand-in for
    the rotating-field cascade of Sec. 8.6.5): gamma 1000, directions uniform in the x-y plane (across the
    laser axis), z ~ U[-lambda/4, lambda/4] about the point where the two pulse fronts meet at t = 0,
    unpolarized (random unit spins).  Both pulses: a0 per component, 1 um, n_cycles sin^2 envelopes
    (field kind CP_COUNTER, phase 0).  NLC and NBW both resolved; photons below photon_store_min (m c^2)
    are not stored.  The beam is generated in chunks of `chunk` electrons, chunk c with seed + c and ids
    c * chunk + i + 1, so any chunk can be made alone."""
    name: str = "cascade_cp2_a500_g1000_n2e8"
    n_electrons: int = 200_000_000
    gamma: float = 1000.0
    a0: float = 500.0
    wavelength_um: float = 1.0
    n_cycles: float = 15.0
    steps: int = 3000
    dt: float = 2.0 * math.pi / 100.0
    photon_store_min: float = 300.0
    seed: int = 5
    chunk: int = 10_000_000

    def instances(self):
        return [{"n": self.n_electrons, "seed": self.seed}]

    def laser(self, inst=None) -> Laser:
        return Laser("CP_COUNTER", self.a0, self.wavelength_um, self.n_cycles, 0.0)

    def chunk_beam(self, c: int, n=None) -> dict:
        """Chunk c of the beam (its first n electrons if n is given)."""
        m = min(self.chunk, self.n_electrons - c * self.chunk) if n is None else n
        rng = np.random.default_rng([self.seed, c])
        pm = math.sqrt(self.gamma * self.gamma - 1.0)
        ph = rng.uniform(0.0, 2.0 * math.pi, m)
        lam = 2.0 * math.pi
        pos = np.zeros((m, 3))
        pos[:, 2] = rng.uniform(-0.25 * lam, 0.25 * lam, m)
        return {"pos": pos, "mom": np.column_stack([pm * np.cos(ph), pm * np.sin(ph), np.zeros(m)]),
                "spin": _unit_vectors(rng, m), "w": np.ones(m),
                "id": np.arange(m, dtype=np.uint64) + np.uint64(c * self.chunk + 1)}

    def n_chunks(self) -> int:
        return (self.n_electrons + self.chunk - 1) // self.chunk

    def sample(self, k: int, inst, m: int) -> dict:
        """m electrons drawn as the beam's are (the growth of a subsample stands for the beam's)."""
        return self.chunk_beam(0, min(m, self.n_electrons))


# 2e8 electrons, gamma 1000, two colliding CP pulses a0 = 500, 1 um, 15 cycles, 3000 steps, NLC + NBW,
# compaction every step, FP32 path; photons below 300 m c^2 not stored.
CASCADE_2E8 = CascadeWorkload()
