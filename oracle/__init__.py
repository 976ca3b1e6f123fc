"""FP64 CPU oracle for the spin- and polarization-resolved strong-field QED step
of Qian et al., arXiv:2511.08929.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never links, loads or calls it, and it shares no code
with the library: it is a plain restatement of the paper (``qed_oracle.c``)
compiled with gcc, plus ctypes marshalling here.

Functions and the equations they follow are documented in ``qed_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import functools
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qed_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# physics flags (same bit meaning as the library's; values restated here from the oracle source)
F_TAU = 1 << 0
F_RECOIL = 1 << 1
F_SPIN_COLLAPSE = 1 << 2
F_POL_COLLAPSE = 1 << 3
F_NONTRANSITION = 1 << 4
F_PUSH = 1 << 5
F_TBMT = 1 << 6
F_TBMT_PAPER = 1 << 7
F_EMIT = 1 << 8
F_RESOLVED = 1 << 9
F_MOVE = 1 << 10
F_SPIN_EVENT = 1 << 11
F_POL_EVENT = 1 << 12
F_AMM = 1 << 13
F_LOOP = 1 << 14
F_G2 = 1 << 15
F_BETA_BASIS = 1 << 16
F_REJECT = 1 << 17
F_MIX_QUANTILE = 1 << 18  # oracle only: emission u' the exact quantile of the spin mixture at r2
F_FULL = (F_TAU | F_RECOIL | F_SPIN_COLLAPSE | F_POL_COLLAPSE | F_NONTRANSITION | F_PUSH | F_TBMT | F_EMIT
          | F_RESOLVED | F_MOVE | F_SPIN_EVENT | F_POL_EVENT)

FIELD_CONST, FIELD_LP, FIELD_CP, FIELD_CP_COUNTER, FIELD_ROT_B = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (FP64, no FMA contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class TableDesc(C.Structure):
    _fields_ = [("chi_min", C.c_double), ("chi_max", C.c_double), ("n_chi", C.c_int32), ("n_r", C.c_int32),
                ("y_lo", C.c_double), ("y_hi", C.c_double)]


class _Tables(C.Structure):
    _fields_ = [("d", TableDesc), ("nlc_rate", C.POINTER(C.c_double)), ("nbw_rate", C.POINTER(C.c_double)),
                ("nlc_icdf", C.POINTER(C.c_double)), ("nbw_icdf", C.POINTER(C.c_double)),
                ("amm", C.POINTER(C.c_double))]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("a0", C.c_double), ("n_cycles", C.c_double),
                ("phase", C.c_double), ("E0", C.c_double * 3), ("B0", C.c_double * 3), ("eta0", C.c_double)]


class Step(C.Structure):
    _fields_ = [("dt", C.c_double), ("t", C.c_double), ("step", C.c_uint64), ("seed", C.c_uint64),
                ("flags", C.c_uint32), ("pad", C.c_uint32), ("photon_store_min", C.c_double),
                ("chi_floor", C.c_double)]


class Counters(C.Structure):
    _fields_ = [("events", C.c_int64), ("stored", C.c_int64), ("dropped_capacity", C.c_int64),
                ("chi_clamped", C.c_int64), ("renormalised", C.c_int64), ("below_store", C.c_int64),
                ("bound_exceeded", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Particles(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_double)) for n in ("x", "y", "z", "px", "py", "pz", "sx", "sy", "sz", "tau", "w")] + [
        ("id", C.POINTER(C.c_uint64)), ("n", C.c_int64), ("capacity", C.c_int64)]


_P = C.POINTER
_D = C.c_double


def lib():
    """Build (if needed) and load the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_philox4x32_10.argtypes = [_P(C.c_uint32), _P(C.c_uint32), _P(C.c_uint32)]
            L.orc_uniform.restype = _D
            L.orc_uniform.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_uniform_pair.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, _P(_D)]
            L.orc_birth_tau.restype = _D
            L.orc_birth_tau.argtypes = [C.c_uint64, C.c_uint64]
            L.orc_child_ids.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, _P(C.c_uint64)]
            L.orc_bessel.argtypes = [_D, _P(_D)]
            L.orc_bessel_scaled.argtypes = [_D, _P(_D)]
            L.orc_nlc_wg.argtypes = [_D, _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D)]
            L.orc_nlc_stokes.argtypes = [_D, _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D)]
            L.orc_nbw_j.argtypes = [_D, _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D)]
            L.orc_nbw_G.argtypes = [_D, _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D)]
            L.orc_rate_integral.restype = _D
            L.orc_rate_integral.argtypes = [C.c_int, _D, C.c_int]
            L.orc_cdf_t.restype = _D
            L.orc_cdf_t.argtypes = [C.c_int, _D, C.c_int, _D]
            L.orc_set_quadrature.restype = C.c_int
            L.orc_set_quadrature.argtypes = [C.c_int, _D]
            L.orc_tables_build.restype = C.c_int
            L.orc_tables_build.argtypes = [_P(TableDesc), _P(_D), _P(_D), _P(_D), _P(_D)]
            for fn in ("orc_nlc_rate_lookup", "orc_nbw_rate_lookup"):
                getattr(L, fn).restype = _D
                getattr(L, fn).argtypes = [_P(_Tables), C.c_int, _D, _P(C.c_int)]
            L.orc_chi.restype = _D
            L.orc_chi.argtypes = [_D, _D, _P(_D), _P(_D), _P(_D)]
            L.orc_airy_scorer.argtypes = [_D, _P(_D)]
            L.orc_amm.restype = _D
            L.orc_amm.argtypes = [_D]
            L.orc_amm_build.restype = C.c_int
            L.orc_amm_build.argtypes = [_P(TableDesc), _P(_D)]
            L.orc_amm_lookup.restype = _D
            L.orc_amm_lookup.argtypes = [_P(_Tables), _D]
            L.orc_icdf_lookup.restype = _D
            L.orc_icdf_lookup.argtypes = [_P(_Tables), C.c_int, C.c_int, _D, _D]
            L.orc_nlc_lambda.restype = _D
            L.orc_nlc_lambda.argtypes = [_D, _D]
            L.orc_nbw_mu.restype = _D
            L.orc_nbw_mu.argtypes = [_D, _D]
            L.orc_field_eval.argtypes = [_P(Field), _P(_D), _D, _P(_D), _P(_D)]
            L.orc_field_eval_n.argtypes = [_P(Field), C.c_int64, _P(_D), _D, _P(_D), _P(_D)]
            L.orc_stokes_to_P.argtypes = [_P(_D)] * 5
            L.orc_P_to_stokes.argtypes = [_P(_D)] * 5
            L.orc_lepton_step.restype = C.c_int
            L.orc_lepton_step.argtypes = [_P(_Tables), _P(Field), _P(Step), C.c_int32, _P(_Particles),
                                          _P(_Particles), _P(Counters)]
            L.orc_photon_step.restype = C.c_int
            L.orc_photon_step.argtypes = [_P(_Tables), _P(Field), _P(Step), _P(_Particles), _P(_Particles),
                                          _P(_Particles), _P(Counters)]
            L.orc_init_tau.argtypes = [_P(_Particles), C.c_uint64]
            L.orc_psi.restype = _D
            L.orc_psi.argtypes = [_D, C.c_int]
            L.orc_mlp_target.argtypes = [_D, _D, _D, _P(_D)]
            L.orc_mlp_cdf.restype = _D
            L.orc_mlp_cdf.argtypes = [_D, _D, _D]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_P(_D))


def _v3(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))
    return a


# ----------------------------------------------------------------------------------------------
# Random numbers (Philox4x32-10) and draws
# ----------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform_pair(pid, seed, step, slot):
    o = (_D * 2)()
    lib().orc_uniform_pair(pid, seed, step, slot, o)
    return o[0], o[1]


def birth_tau(pid, seed):
    return lib().orc_birth_tau(pid, seed)


def child_ids(pid, seed, step):
    o = (C.c_uint64 * 2)()
    lib().orc_child_ids(pid, seed, step, o)
    return int(o[0]), int(o[1])


# ----------------------------------------------------------------------------------------------
# Bessel functions and spectra
# ----------------------------------------------------------------------------------------------
def bessel(x, scaled=False):
    """(K_{1/3}(x), K_{2/3}(x), int_x^inf K_{1/3}); times e^x if scaled."""
    o = (_D * 3)()
    (lib().orc_bessel_scaled if scaled else lib().orc_bessel)(float(x), o)
    return np.array(o[:])


def nlc_wg(lam, bes, si, eps, beta, k):
    w = _D()
    g = np.zeros(3)
    b = np.ascontiguousarray(bes, dtype=np.float64)
    lib().orc_nlc_wg(lam, _dp(b), _dp(_v3(si)), _dp(_v3(eps)), _dp(_v3(beta)), _dp(_v3(k)), C.byref(w), _dp(g))
    return w.value, g


def nlc_stokes(lam, bes, si, sf, eps, beta, k):
    F = np.zeros(4)
    b = np.ascontiguousarray(bes, dtype=np.float64)
    lib().orc_nlc_stokes(lam, _dp(b), _dp(_v3(si)), _dp(_v3(sf)), _dp(_v3(eps)), _dp(_v3(beta)), _dp(_v3(k)), _dp(F))
    return F


def nbw_j(lam, bes, xi, eps, beta, k):
    w0 = _D()
    je = np.zeros(3)
    jp = np.zeros(3)
    b = np.ascontiguousarray(bes, dtype=np.float64)
    lib().orc_nbw_j(lam, _dp(b), _dp(_v3(xi)), _dp(_v3(eps)), _dp(_v3(beta)), _dp(_v3(k)), C.byref(w0), _dp(je),
                    _dp(jp))
    return w0.value, je, jp


def nbw_G(lam, bes, sp, se, eps, beta, k):
    G = np.zeros(4)
    b = np.ascontiguousarray(bes, dtype=np.float64)
    lib().orc_nbw_G(lam, _dp(b), _dp(_v3(sp)), _dp(_v3(se)), _dp(_v3(eps)), _dp(_v3(beta)), _dp(_v3(k)), _dp(G))
    return G


def rate_integral(nbw: bool, chi: float, sigma: int) -> float:
    """NLC: int_0^1 w_sigma d lambda.  NBW: same, scaled by e^{8/(3 chi)}."""
    return lib().orc_rate_integral(int(nbw), float(chi), int(sigma))


def cdf_t(nbw: bool, chi: float, sigma: int, t: float) -> float:
    return lib().orc_cdf_t(int(nbw), float(chi), int(sigma), float(t))


def set_quadrature(n_points: int, width: float):
    if lib().orc_set_quadrature(int(n_points), float(width)) != 0:
        raise ValueError("bad quadrature rule")


def psi(chi: float, which: int) -> float:
    return lib().orc_psi(float(chi), int(which))


def mlp_target(chi: float, r: float, s: float):
    """(ln u', xi1, xi2, xi3): the exact r-quantile of the NLC spectrum with spin projection s and the
    photon Stokes vector there (final spin summed) -- the learned sampler's target."""
    out = (_D * 4)()
    lib().orc_mlp_target(float(chi), float(r), float(s), out)
    return np.array(out[:])


def mlp_cdf(chi: float, s: float, ln_up: float) -> float:
    """Exact mixture CDF of the NLC spectrum with spin projection s at u' = exp(ln_up)."""
    return lib().orc_mlp_cdf(float(chi), float(s), float(ln_up))


def chi(eta0, e, p, E, B):
    """chi of a particle of energy e, momentum p in E, B, as the step functions evaluate it."""
    return lib().orc_chi(float(eta0), float(e), _dp(_v3(p)), _dp(_v3(E)), _dp(_v3(B)))


def airy_scorer(z: float):
    """(Ai(z), Gi(z)) for z >= 0 from the integral definition (App. A.1)."""
    out = np.zeros(2)
    lib().orc_airy_scorer(float(z), _dp(out))
    return float(out[0]), float(out[1])


def amm(chi: float) -> float:
    """Field-dependent anomalous moment a(chi) (one-loop Scorer term), by quadrature."""
    return lib().orc_amm(float(chi))


def nlc_lambda(chi, up):
    return lib().orc_nlc_lambda(chi, up)


def nbw_mu(chi, x):
    return lib().orc_nbw_mu(chi, x)


def stokes_to_P(xi, eps, beta, k):
    P = np.zeros(3)
    lib().orc_stokes_to_P(_dp(_v3(xi)), _dp(_v3(eps)), _dp(_v3(beta)), _dp(_v3(k)), _dp(P))
    return P


def P_to_stokes(P, eps, beta, k):
    xi = np.zeros(3)
    lib().orc_P_to_stokes(_dp(_v3(P)), _dp(_v3(eps)), _dp(_v3(beta)), _dp(_v3(k)), _dp(xi))
    return xi


# ----------------------------------------------------------------------------------------------
# Tables
# ----------------------------------------------------------------------------------------------
class Tables:
    """Oracle-built rate and ICDF tables (see orc_tables_build)."""

    def __init__(self, chi_min=1e-4, chi_max=1e3, n_chi=256, n_r=256, y_lo=-20.0, y_hi=20.0):
        self.desc = TableDesc(chi_min, chi_max, n_chi, n_r, y_lo, y_hi)
        self.nlc_rate = np.zeros((2, n_chi))
        self.nbw_rate = np.zeros((2, n_chi))
        self.nlc_icdf = np.zeros((2, n_chi, n_r))
        self.nbw_icdf = np.zeros((2, n_chi, n_r))
        rc = lib().orc_tables_build(C.byref(self.desc), _dp(self.nlc_rate), _dp(self.nbw_rate), _dp(self.nlc_icdf),
                                    _dp(self.nbw_icdf))
        if rc != 0:
            raise ValueError("bad table description")
        self._s = _Tables(self.desc, _dp(self.nlc_rate), _dp(self.nbw_rate), _dp(self.nlc_icdf),
                          _dp(self.nbw_icdf), None)
        self.amm = None

    def ensure_amm(self):
        """Build the ln a(chi) table on the rate grid (needed by the F_AMM and F_LOOP steps)."""
        if self.amm is None:
            amm = np.zeros(self.desc.n_chi)
            if lib().orc_amm_build(C.byref(self.desc), _dp(amm)) != 0:
                raise ValueError("bad table description")
            self.amm = amm
            self._s.amm = _dp(self.amm)
        return self

    def amm_lookup(self, chi):
        return lib().orc_amm_lookup(self.ref, chi)

    @property
    def ref(self):
        return C.byref(self._s)

    def nlc_rate_lookup(self, s, chi):
        return lib().orc_nlc_rate_lookup(self.ref, s, chi, None)

    def nbw_rate_lookup(self, s, chi):
        return lib().orc_nbw_rate_lookup(self.ref, s, chi, None)

    def icdf(self, nbw, s, chi, r):
        return lib().orc_icdf_lookup(self.ref, int(nbw), s, chi, r)


@functools.lru_cache(maxsize=8)
def tables(chi_min=1e-4, chi_max=1e3, n_chi=256, n_r=256, y_lo=-20.0, y_hi=20.0) -> Tables:
    return Tables(chi_min, chi_max, n_chi, n_r, y_lo, y_hi)


# ----------------------------------------------------------------------------------------------
# Fields and particles
# ----------------------------------------------------------------------------------------------
def field(kind=FIELD_LP, a0=0.0, n_cycles=10.0, phase=0.0, E0=(0, 0, 0), B0=(0, 0, 0), eta0=3.0329e-6) -> Field:
    f = Field()
    f.kind = kind
    f.a0 = a0
    f.n_cycles = n_cycles
    f.phase = phase
    for i in range(3):
        f.E0[i] = E0[i]
        f.B0[i] = B0[i]
    f.eta0 = eta0
    return f


def field_eval(f: Field, x, t):
    E = np.zeros(3)
    B = np.zeros(3)
    lib().orc_field_eval(C.byref(f), _dp(_v3(x)), float(t), _dp(E), _dp(B))
    return E, B


def field_eval_n(f: Field, x, t):
    """Fields at the rows of x (n, 3) at time t: (E, B), each (n, 3)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))
    E = np.zeros_like(x)
    B = np.zeros_like(x)
    lib().orc_field_eval_n(C.byref(f), len(x), _dp(x), float(t), _dp(E), _dp(B))
    return E, B


def step_desc(dt, t, step, seed, flags=F_FULL, photon_store_min=0.0, chi_floor=0.0) -> Step:
    s = Step()
    s.dt = dt
    s.t = t
    s.step = step
    s.seed = seed
    s.flags = flags
    s.photon_store_min = photon_store_min
    s.chi_floor = chi_floor
    return s


COLS = ("x", "y", "z", "px", "py", "pz", "sx", "sy", "sz", "tau", "w")


class Particles:
    """FP64 structure-of-arrays particle buffer with a fixed capacity.
    For photons (px, py, pz) is the momentum k and (sx, sy, sz) the polarization vector P."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        cap = max(self.capacity, 1)
        self.a = {c: np.zeros(cap) for c in COLS}
        self.id = np.zeros(cap, dtype=np.uint64)
        self._s = _Particles(*[_dp(self.a[c]) for c in COLS], self.id.ctypes.data_as(_P(C.c_uint64)), 0,
                             self.capacity)

    @classmethod
    def from_arrays(cls, capacity, pos, mom, spin, w, ids, tau=None):
        p = cls(capacity)
        n = len(ids)
        if n > capacity:
            raise ValueError("capacity")
        for j, c in enumerate(("x", "y", "z")):
            p.a[c][:n] = pos[:, j]
        for j, c in enumerate(("px", "py", "pz")):
            p.a[c][:n] = mom[:, j]
        for j, c in enumerate(("sx", "sy", "sz")):
            p.a[c][:n] = spin[:, j]
        p.a["w"][:n] = w
        p.id[:n] = ids
        if tau is not None:
            p.a["tau"][:n] = tau
        p._s.n = n
        return p

    @property
    def n(self):
        return int(self._s.n)

    @property
    def ref(self):
        return C.byref(self._s)

    def init_tau(self, seed):
        lib().orc_init_tau(self.ref, seed)

    def view(self):
        n = self.n
        d = {c: self.a[c][:n].copy() for c in COLS}
        d["id"] = self.id[:n].copy()
        d["pos"] = np.stack([d["x"], d["y"], d["z"]], 1)
        d["mom"] = np.stack([d["px"], d["py"], d["pz"]], 1)
        d["spin"] = np.stack([d["sx"], d["sy"], d["sz"]], 1)
        return d


def lepton_step(tb: Tables, f: Field, st: Step, charge: int, leptons: Particles, photons: Particles | None,
                ctr: Counters | None = None) -> Counters:
    ctr = ctr if ctr is not None else Counters()
    rc = lib().orc_lepton_step(tb.ref, C.byref(f), C.byref(st), int(charge), leptons.ref,
                               photons.ref if photons is not None else None, C.byref(ctr))
    if rc == -2:
        raise ValueError("flags need the a(chi) table (Tables.ensure_amm) or contradict each other")
    if rc != 0:
        raise MemoryError("oracle lepton step failed")
    return ctr


def photon_step(tb: Tables, f: Field, st: Step, photons: Particles, electrons: Particles | None,
                positrons: Particles | None, ctr: Counters | None = None) -> Counters:
    ctr = ctr if ctr is not None else Counters()
    rc = lib().orc_photon_step(tb.ref, C.byref(f), C.byref(st), photons.ref,
                               electrons.ref if electrons is not None else None,
                               positrons.ref if positrons is not None else None, C.byref(ctr))
    if rc != 0:
        raise MemoryError("oracle photon step failed")
    return ctr


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int):
    lib().orc_set_num_threads(int(n))


__all__ = [n for n in dir(sys.modules[__name__]) if not n.startswith("_")]
