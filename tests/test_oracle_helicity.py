"""The helicity-transfer benchmarks of Sec. 8.6.3 and 8.6.4 in their plane-wave analogues, on the oracle
(CPU): 10 GeV electrons of helicity +1 (6 % spread) against a linearly polarized pulse (a0 = 50) emit
photons whose circular polarization rises with energy to nearly 100 % (X14), and against a circularly
polarized pulse (a0 = 100) make positrons whose longitudinal polarization rises with energy to nearly
100 % (X15).  Flipping the electrons' helicity flips both signs; unpolarized electrons give none."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2511_08929_gb300 import inputs as I

from parity_util import oracle_full_step

GEV = 1e9 / I.ME_EV


@pytest.fixture(scope="module")
def tb():
    return O.tables(1e-3, 1e2, 64, 128)


def _run(tb, wl, n, spin_dir=None, spin="fixed", pairs=True):
    w = dataclasses.replace(wl, n_electrons=n, spin=spin, spin_dir=spin_dir or wl.spin_dir)
    b = w.beam()
    E = O.Particles.from_arrays(20 * n, b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    E.init_tau(w.seed)
    P, G = O.Particles(20 * n), O.Particles(100 * n)
    f = O.field({"LP": O.FIELD_LP, "CP": O.FIELD_CP}[w.laser.kind], a0=w.laser.a0, n_cycles=w.laser.n_cycles,
                eta0=w.laser.eta0)
    for s in range(w.crossing_steps()):
        st = O.step_desc(w.dt, s * w.dt, s, w.seed, O.F_FULL)
        if pairs:
            oracle_full_step(tb, f, st, [(E, -1), (P, 1)], G, E, P)
        else:
            O.lepton_step(tb, f, st, -1, E, G)
    return E, P, G


def _binned(mom, vec, lepton):
    e = np.linalg.norm(mom, axis=1)
    en = np.sqrt(1.0 + e * e) if lepton else e
    comp = (vec * mom).sum(1) / e
    idx = np.floor(en / GEV).astype(int)
    means = np.array([comp[idx == i].mean() if np.any(idx == i) else np.nan for i in range(10)])
    counts = np.array([np.sum(idx == i) for i in range(10)])
    return means, counts


def test_x14_circular_polarization_rises_with_energy(tb):
    _, _, G = _run(tb, I.HELICITY_LP_X14, 2000, pairs=False)
    v = G.view()
    m, c = _binned(v["mom"], v["spin"], False)
    assert G.n > 10000
    assert abs(m[0]) < 0.1  # soft photons: nearly unpolarized
    assert np.all(np.diff(m[1:7]) > 0)  # rising through the spectrum
    top = (c[7:] * m[7:]).sum() / c[7:].sum()
    assert top > 0.85, m
    # helicity -1: the same with the opposite sign; unpolarized electrons: none
    _, _, G2 = _run(tb, I.HELICITY_LP_X14, 2000, spin_dir=(0.0, 0.0, 1.0), pairs=False)
    m2, c2 = _binned(G2.view()["mom"], G2.view()["spin"], False)
    assert (c2[7:] * m2[7:]).sum() / c2[7:].sum() < -0.85
    _, _, G3 = _run(tb, I.HELICITY_LP_X14, 2000, spin="random", pairs=False)
    v3 = G3.view()
    m3, c3 = _binned(v3["mom"], v3["spin"], False)
    hi = c3[3:].sum()
    assert abs((c3[3:] * np.nan_to_num(m3[3:])).sum() / hi) < 4.0 / math.sqrt(hi)


def test_x15_positron_longitudinal_polarization_rises_with_energy(tb):
    _, P, _ = _run(tb, I.HELICITY_CP_X15, 3000)
    v = P.view()
    m, c = _binned(v["mom"], v["spin"], True)
    assert P.n > 1000
    assert abs(m[0]) < 0.1
    assert m[1] < m[2] < m[3]
    top = (c[4:] * np.nan_to_num(m[4:])).sum() / c[4:].sum()
    assert top > 0.65, m
    _, P2, _ = _run(tb, I.HELICITY_CP_X15, 3000, spin_dir=(0.0, 0.0, 1.0))
    m2, c2 = _binned(P2.view()["mom"], P2.view()["spin"], True)
    assert (c2[4:] * np.nan_to_num(m2[4:])).sum() / c2[4:].sum() < -0.65
