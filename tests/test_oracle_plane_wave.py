"""The plane-wave identities the FP32 path relies on, checked on the oracle's fields (CPU).

The FP32 kernels evaluate chi and the basis vector f = E + v x B in reduced forms for the linear and
circular lasers, and drop the products by E_z and B_z in the Boris push and the T-BMT vector for every
plane-wave kind.  These hold when the field is transverse (E_z = B_z = 0) and, for the reduced chi and
f, when it is a single wave along +z (B = z x E):

  chi = eta0 sqrt((e E + p x B)^2 - (p.E)^2)  =  eta0 |e - p_z| |E|          (Sec. 1, the invariant)
  f   = E + v x B                              =  (1 - v_z) E + (v.E) z

Here they are checked against the oracle's own field evaluation at random points and times, with the
general forms written out in NumPy, so that a field kind whose fields break an assumption fails here.
"""
import numpy as np
import pytest

import oracle as O

ETA0 = 3.0329e-6


def _points(rng, n):
    x = rng.uniform(-40.0, 40.0, (n, 3))
    t = rng.uniform(0.0, 80.0, n)
    return x, t


def _chi_general(e, p, E, B):
    a = e * E + np.cross(p, B)
    v = a @ a - (p @ E) ** 2
    return ETA0 * np.sqrt(max(v, 0.0))


@pytest.mark.parametrize("kind", [O.FIELD_LP, O.FIELD_CP])
def test_single_wave_fields_are_z_cross_E(kind):
    rng = np.random.default_rng(3 + kind)
    f = O.field(kind, a0=120.0, n_cycles=4.0, phase=0.7)
    x, t = _points(rng, 400)
    seen = 0
    for xi, ti in zip(x, t):
        E, B = O.field_eval(f, xi, ti)
        assert E[2] == 0.0 and B[2] == 0.0
        np.testing.assert_allclose(B, np.cross([0.0, 0.0, 1.0], E), rtol=0, atol=1e-12 * (1.0 + abs(E).max()))
        seen += np.any(E != 0.0)
    assert seen > 50  # the points sample the pulse, not only the empty space around it


def test_counter_propagating_fields_are_transverse():
    rng = np.random.default_rng(11)
    f = O.field(O.FIELD_CP_COUNTER, a0=80.0, n_cycles=4.0)
    x, t = _points(rng, 400)
    off = 0
    for xi, ti in zip(x, t):
        E, B = O.field_eval(f, xi, ti)
        assert E[2] == 0.0 and B[2] == 0.0
        off += not np.allclose(B, np.cross([0.0, 0.0, 1.0], E), atol=1e-9)
    assert off > 0  # two waves: B is not z x E, so the reduced chi and f must not be used here


@pytest.mark.parametrize("kind", [O.FIELD_LP, O.FIELD_CP])
def test_reduced_chi_and_basis_vector(kind):
    rng = np.random.default_rng(17 + kind)
    f = O.field(kind, a0=150.0, n_cycles=4.0, phase=0.3)
    x, t = _points(rng, 300)
    for xi, ti in zip(x, t):
        E, B = O.field_eval(f, xi, ti)
        # a lepton (e = gamma) and a photon (e = |k|) moving in arbitrary directions, head-on included
        for massive in (True, False):
            p = rng.normal(size=3) * rng.uniform(1.0, 5000.0)
            if rng.uniform() < 0.3:
                p = np.array([0.0, 0.0, -abs(p[2]) - 1.0])
            e = np.sqrt(1.0 + p @ p) if massive else np.sqrt(p @ p)
            chi = _chi_general(e, p, E, B)
            red = ETA0 * abs(e - p[2]) * np.hypot(E[0], E[1])
            assert red == pytest.approx(chi, rel=1e-9, abs=1e-300)
            v = p / e
            fg = E + np.cross(v, B)
            fr = np.array([(1.0 - v[2]) * E[0], (1.0 - v[2]) * E[1], v[0] * E[0] + v[1] * E[1]])
            np.testing.assert_allclose(fr, fg, rtol=1e-12, atol=1e-12 * (1.0 + abs(E).max()))


def test_reduced_chi_fails_for_the_counter_propagating_field():
    """A guard on the guard: the reduced form is wrong for two waves, so the tests above can fail."""
    rng = np.random.default_rng(5)
    f = O.field(O.FIELD_CP_COUNTER, a0=80.0, n_cycles=4.0)
    worst = 0.0
    for xi, ti in zip(*_points(rng, 300)):
        E, B = O.field_eval(f, xi, ti)
        if not np.any(E):
            continue
        p = np.array([0.0, 0.0, -2000.0])
        e = np.sqrt(1.0 + p @ p)
        chi = _chi_general(e, p, E, B)
        red = ETA0 * abs(e - p[2]) * np.hypot(E[0], E[1])
        worst = max(worst, abs(red - chi) / max(chi, 1e-300))
    assert worst > 1e-3


def _chi_mp(e, p, E, B, m2):
    """The invariant of Sec. 1 in 60-digit arithmetic from the same (double) inputs; e recomputed from p."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    P = [mp.mpf(float(x)) for x in p]
    Ev = [mp.mpf(float(x)) for x in E]
    Bv = [mp.mpf(float(x)) for x in B]
    ee = mp.sqrt(m2 + sum(x * x for x in P))
    pxB = [P[1] * Bv[2] - P[2] * Bv[1], P[2] * Bv[0] - P[0] * Bv[2], P[0] * Bv[1] - P[1] * Bv[0]]
    a = [ee * Ev[i] + pxB[i] for i in range(3)]
    pe = sum(P[i] * Ev[i] for i in range(3))
    return float(ETA0 * mp.sqrt(sum(x * x for x in a) - pe * pe))


@pytest.mark.parametrize("kind", [O.FIELD_CP, O.FIELD_CP_COUNTER])
def test_chi_evaluation_against_60_digits(kind):
    """The oracle's chi against the invariant in 60-digit arithmetic from the same inputs: generic
    directions to 1e-13; leptons and photons moving with the forward wave (angles 1e-4 .. 1e-2 to it,
    gamma 1e2 .. 1e4) to 4e-16 x the cancellation factor (e|E| + |p||B|)^2 / (chi/eta0)^2 of the formula
    (both inside e E + p x B and in the difference of squares), which for an angle theta to the wave grows
    like 16/theta^4: the invariant itself is that ill-conditioned for such particles in double."""
    rng = np.random.default_rng(11 + kind)
    f = O.field(kind, a0=200.0, n_cycles=4.0, phase=0.7)
    n_checked = 0
    for xi, ti in zip(*_points(rng, 200)):
        E, B = O.field_eval(f, xi, ti)
        if not np.any(E):
            continue
        for m2 in (1.0, 0.0):
            p = rng.normal(size=3) * rng.uniform(1.0, 5000.0)  # generic
            e = np.sqrt(m2 + p @ p)
            assert O.chi(ETA0, e, p, E, B) == pytest.approx(_chi_mp(e, p, E, B, m2), rel=1e-13)
            th = 10 ** rng.uniform(-4, -2)  # co-moving with the forward wave
            g = 10 ** rng.uniform(2, 4)
            ph = rng.uniform(0, 2 * np.pi)
            p = g * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
            e = np.sqrt(m2 + p @ p)
            ref = _chi_mp(e, p, E, B, m2)
            kappa = (e * np.linalg.norm(E) + np.linalg.norm(p) * np.linalg.norm(B)) ** 2 / max((ref / ETA0) ** 2, 1e-300)
            got = O.chi(ETA0, e, p, E, B)
            assert abs(got - ref) <= 4e-16 * kappa * ref + 1e-300, (got, ref, kappa)
            n_checked += 1
    assert n_checked > 50
