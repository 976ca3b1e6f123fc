"""Pins of the oracle's one-loop terms (App. A.1) and the field-dependent anomalous moment g(chi)
(Sec. 8.6.2), CPU only.

* Ai and Gi from the integral definition Ai(z) + i Gi(z) = (1/pi) int_0^inf exp(i(zt + t^3/3)) dt
  against mpmath's Scorer function and scipy's Airy function (independent libraries).
* a(chi) = (alpha/chi) int dlambda lambda Gi(z)/sqrt(z): Schwinger's alpha/(2 pi) at chi -> 0, the
  closed-form large-chi asymptote alpha Gi(0) B(5/3, 4/3) chi^{-2/3} with Gi(0) = 1/(3^{7/6} Gamma(2/3)),
  and mpmath's adaptive quadrature of the u-form of the same integral.
* The T-BMT step with g(chi) reduces to the constant-moment step in weak fields; with g = 2 the spin
  keeps its angle to the momentum in a pure magnetic field up to the Boris push's phase error (closed
  form); the loop's Scorer term in the no-emission update turns the spin as T-BMT's anomalous part with
  a(chi) does in a crossed field (where the rest-frame |B'| = |E'| = chi/eta0), so the two routes agree
  to the splitting error of applying the two turns one after the other, first order in dt.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2511_08929_gb300 import inputs as I

mp = pytest.importorskip("mpmath")
sp = pytest.importorskip("scipy.special")

ALPHA = 7.2973525693e-3
A0 = ALPHA / (2 * math.pi)
ETA0 = I.eta0_for_wavelength(0.8)


@pytest.mark.parametrize("z", [0.0, 1e-3, 0.1, 0.5, 1.0, 2.0, 3.7, 10.0, 55.0, 300.0, 1e4])
def test_scorer_gi_against_mpmath(z):
    ai, gi = O.airy_scorer(z)
    assert gi == pytest.approx(float(mp.scorergi(z)), rel=1e-13)
    ref_ai = sp.airy(z)[0]
    if z <= 4.0:
        assert ai == pytest.approx(ref_ai, rel=1e-12)
    assert abs(ai - ref_ai) < 1e-15  # Ai from the same integral: absolute accuracy only


def test_scorer_at_zero_closed_form():
    """Gi(0) = Ai(0)/sqrt(3) = 1/(3^{7/6} Gamma(2/3)) (DLMF 9.12.4)."""
    ai, gi = O.airy_scorer(0.0)
    g23 = math.gamma(2.0 / 3.0)
    assert gi == pytest.approx(1.0 / (3 ** (7 / 6) * g23), rel=1e-14)
    assert ai == pytest.approx(1.0 / (3 ** (2 / 3) * g23), rel=1e-14)


def test_amm_schwinger_limit():
    """a(chi) -> alpha/(2 pi) as chi -> 0, from below, with the deficit shrinking faster than chi."""
    r = [O.amm(c) / A0 for c in (1e-5, 1e-4, 1e-3, 1e-2)]
    assert r[0] == pytest.approx(1.0, abs=2e-8)
    assert all(x < 1.0 for x in r)
    d = [1.0 - x for x in r]
    assert d[1] < 0.02 * d[2] and d[2] < 0.02 * d[3]


def test_amm_large_chi_asymptote():
    """a(chi) chi^{2/3} -> alpha Gi(0) B(5/3, 4/3) with Gi(0) = 1/(3^{7/6} Gamma(2/3)), approached from
    above with a relative excess that falls roughly as chi^{-2/3}."""
    gi0 = 1.0 / (3 ** (7 / 6) * math.gamma(2.0 / 3.0))
    B = math.gamma(5.0 / 3.0) * math.gamma(4.0 / 3.0) / math.gamma(3.0)
    lim = ALPHA * gi0 * B
    ex = [O.amm(c) * c ** (2 / 3) / lim - 1.0 for c in (1e4, 1e6, 1e8)]
    assert ex[2] == pytest.approx(0.0, abs=2e-5)
    assert ex[0] > ex[1] > ex[2] > 0.0
    assert ex[1] < 0.1 * ex[0] and ex[2] < 0.1 * ex[1]


@pytest.mark.parametrize("chi", [0.05, 1.0, 30.0])
def test_amm_against_mpmath_u_form(chi):
    """a(chi) = (alpha/chi) int_0^inf du u/(1+u)^3 Gi(z)/sqrt(z), z = (u/chi)^{2/3}, by mpmath's quadrature
    with mpmath's Scorer function (an independent representation and library)."""
    mp.mp.dps = 20
    f = lambda u: u / (1 + u) ** 3 * mp.scorergi((u / chi) ** (mp.mpf(2) / 3)) / (u / chi) ** (mp.mpf(1) / 3)
    ref = ALPHA / chi * mp.quad(f, [0, chi / 10, chi, 10 * chi, 100 * chi, mp.inf])
    assert O.amm(chi) == pytest.approx(float(ref), rel=1e-12)


def test_amm_table_lookup(small_tables):
    tb = small_tables.ensure_amm()
    d = tb.desc
    chis = np.exp(np.linspace(math.log(d.chi_min), math.log(d.chi_max), d.n_chi))
    for c in chis[[0, 3, d.n_chi // 2, -1]]:
        assert tb.amm_lookup(c) == pytest.approx(O.amm(c), rel=1e-12)
    assert tb.amm_lookup(d.chi_min * 1e-3) == tb.amm_lookup(d.chi_min)
    assert tb.amm_lookup(d.chi_max * 1e3) == tb.amm_lookup(d.chi_max)
    assert np.all(np.diff(tb.amm) < 0)  # a(chi) falls monotonically
    # between nodes: linear in (ln chi, ln a)
    m = math.sqrt(chis[5] * chis[6])
    assert math.log(tb.amm_lookup(m)) == pytest.approx(0.5 * (tb.amm[5] + tb.amm[6]), rel=1e-13)


def _one(p, s, pid=1):
    return {"pos": np.zeros((1, 3)), "mom": np.array([p], float), "spin": np.array([s], float), "w": np.ones(1),
            "id": np.array([pid], dtype=np.uint64)}


def _run(tb, b, f, flags, n, dt, q=-1, tau=None):
    L = O.Particles.from_arrays(1, b["pos"], b["mom"], b["spin"], b["w"], b["id"],
                                tau=None if tau is None else np.array([tau]))
    for k in range(n):
        O.lepton_step(tb, f, O.step_desc(dt, k * dt, k, 3, flags), q, L, None)
    return L.view()


def test_g_of_chi_weak_field_is_constant_moment(small_tables):
    """chi ~ 1e-6, below the table's grid: the g(chi) step takes a(chi_min), so it differs from the
    alpha/(2 pi) step by (a(chi_min)/a0 - 1) times the whole anomalous turn (the g = 2 step's difference)."""
    tb = small_tables.ensure_amm()
    g, Bz, dt, n = 50.0, 1e-2, 0.05, 200
    pm = math.sqrt(g * g - 1)
    b = _one([pm, 0, 0], [1.0, 0, 0])
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    base = O.F_PUSH | O.F_TBMT | O.F_MOVE
    s0 = _run(tb, b, f, base, n, dt)["spin"][0]
    s1 = _run(tb, b, f, base | O.F_AMM, n, dt)["spin"][0]
    s2 = _run(tb, b, f, base | O.F_G2, n, dt)["spin"][0]
    assert np.abs(s2 - s0).max() > 1e-6  # the moment itself is visible at this size
    k = tb.amm_lookup(tb.desc.chi_min) / A0 - 1.0
    assert -1e-4 < k < 0
    d = s1 - s0
    assert np.linalg.norm(d - k * (s0 - s2)) < 1e-3 * np.linalg.norm(d)


def test_g2_spin_follows_momentum_in_magnetic_field(small_tables):
    """g = 2, E = 0: s turns by B dt/gamma_bar per step and p by 2 atan(B dt/(2 gamma)), so the angle
    between them changes by the closed-form difference only (no anomalous precession)."""
    tb = small_tables
    g, Bz, dt, n = 50.0, 10.0, 0.05, 400
    pm = math.sqrt(g * g - 1)
    b = _one([pm, 0, 0], [1.0, 0, 0], pid=3)
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    v = _run(tb, b, f, O.F_PUSH | O.F_TBMT | O.F_MOVE | O.F_G2, n, dt)
    th_p = 2 * math.atan(Bz * dt / (2 * g))
    gbar = math.sqrt(1 + (pm * math.cos(th_p / 2)) ** 2)
    exact = n * (Bz * dt / gbar - th_p)
    rel = math.atan2(v["spin"][0][1], v["spin"][0][0]) - math.atan2(v["mom"][0][1], v["mom"][0][0])
    rel = (rel + math.pi) % (2 * math.pi) - math.pi
    assert rel == pytest.approx(exact, abs=1e-11)
    assert abs(exact) < 1e-3  # and that is far below the anomalous precession a B t = 0.023


def _crossed(E0):
    """A constant crossed field (E perpendicular to B, |E| = |B|), the plane-wave case: wave along +z."""
    return O.field(O.FIELD_CONST, E0=(E0, 0, 0), B0=(0, E0, 0), eta0=ETA0)


def test_loop_scorer_term_equals_g_of_chi_in_crossed_field(small_tables):
    """Head-on 500 MeV electron in a crossed field with chi ~ 0.5, events suppressed by a huge optical
    depth: T-BMT with g(chi) (F_AMM) and T-BMT with g = 2 plus the loop's Scorer term in the no-emission
    update (F_LOOP) give the same spin to the splitting error (first order: it halves with dt), while
    both differ from g = 2 alone by the anomalous precession."""
    tb = small_tables.ensure_amm()
    g = 1000.0
    pz = -math.sqrt(g * g - 1)
    E0 = 0.5 / (ETA0 * 2 * g)  # chi = eta0 gamma (1 + beta) E0
    b = _one([0, 0, pz], [0.6, 0.0, 0.8], pid=5)
    f = _crossed(E0)
    base = O.F_PUSH | O.F_TBMT | O.F_MOVE | O.F_EMIT | O.F_TAU
    T = 40.0
    diffs = []
    for dt in (0.02, 0.01):
        n = int(round(T / dt))
        sa = _run(tb, b, f, base | O.F_AMM, n, dt, tau=1e300)["spin"][0]
        sl = _run(tb, b, f, base | O.F_LOOP, n, dt, tau=1e300)["spin"][0]
        s2 = _run(tb, b, f, base | O.F_G2, n, dt, tau=1e300)["spin"][0]
        eff = np.linalg.norm(sa - s2)
        assert eff > 0.05  # the anomalous precession turns the spin visibly
        diffs.append(np.linalg.norm(sl - sa))
        assert diffs[-1] < 2e-3 * eff
    assert 0.4 * diffs[0] < diffs[1] < 0.6 * diffs[0]


def test_loop_sense_for_positrons(small_tables):
    """No push: every turn is about y (B = E0 y, beta x E = -E0 y for the head-on lepton), so the
    anomalous turn is the angle in the (z, x) plane between the g(chi) (or loop) spin and the g = 2 spin.
    The loop's turn equals g(chi)'s for either charge, and a positron turns the opposite way to an
    electron (T-BMT sense -q)."""
    tb = small_tables.ensure_amm()
    g = 1000.0
    pz = -math.sqrt(g * g - 1)
    E0 = 0.5 / (ETA0 * 2 * g)
    f = _crossed(E0)
    b = _one([0, 0, pz], [0.6, 0.0, 0.8], pid=7)
    base = O.F_TBMT | O.F_EMIT | O.F_TAU
    dt, n = 0.01, 2000
    ang = {}
    for q in (-1, 1):
        for fl in (O.F_AMM, O.F_LOOP, O.F_G2):
            s_ = _run(tb, b, f, base | fl, n, dt, q=q, tau=1e300)["spin"][0]
            assert abs(s_[1]) < 1e-14
            ang[q, fl] = math.atan2(s_[0], s_[2])
    turn = {k: (ang[k] - ang[k[0], O.F_G2] + math.pi) % (2 * math.pi) - math.pi for k in ang}
    assert abs(turn[-1, O.F_AMM]) > 0.05
    for q in (-1, 1):
        assert turn[q, O.F_LOOP] == pytest.approx(turn[q, O.F_AMM], rel=2e-3)
    assert turn[1, O.F_AMM] == pytest.approx(-turn[-1, O.F_AMM], rel=1e-9)


def test_flag_errors(small_tables):
    f = _crossed(1.0)
    b = _one([0, 0, -100.0], [0, 0, 1.0])
    L = O.Particles.from_arrays(1, b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    tb_plain = O.Tables(1e-3, 10.0, 8, 16)
    with pytest.raises(ValueError):
        O.lepton_step(tb_plain, f, O.step_desc(0.1, 0, 0, 1, O.F_TBMT | O.F_AMM), -1, L, None)
    tb = small_tables.ensure_amm()
    for bad in (O.F_AMM | O.F_G2, O.F_AMM | O.F_LOOP):
        with pytest.raises(ValueError):
            O.lepton_step(tb, f, O.step_desc(0.1, 0, 0, 1, O.F_TBMT | bad), -1, L, None)
