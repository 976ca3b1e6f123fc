"""The two spin-evolution benchmarks of Sec. 8.3 reduced to 0-D with analytic fields, CPU only: the
oracle's Monte Carlo ensemble against the extended Baier-Katkov-Strakhovenko equation

    dS/dt = Omega x S - Gamma [psi1 S + psi2 (S.v) v - psi3 beta],   Gamma = alpha/(sqrt3 pi eta0 gamma),

integrated here by RK4 together with the classical orbit (Omega the standard T-BMT vector, beta the
basis vector of the spin quantization, psi from the oracle's quadrature, which is pinned against scipy
elsewhere; the sign of the psi3 term is that of the Sokolov-Ternov closed form, pinned there too).

* X7: a 1 GeV electron beam polarized along x gyrating in a constant B along z at chi = 1.  With the
  spin quantization axis (SQA) every component follows the equation; with spins resolved along +-beta
  only, the component along B still does, the transverse ones decay too fast (each emission projects
  them out).
* X8: an unpolarized beam whose field turns from z to y at about the gyrofrequency after the beam has
  polarized along -z: the SQA ensemble follows the equation through and after the turn; the beta-basis
  ensemble leaves it once the field has turned.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2511_08929_gb300 import inputs as I

ALPHA = 7.2973525693e-3
AE = ALPHA / (2 * math.pi)
ETA0 = I.eta0_for_wavelength(0.8)
GAMMA_1GEV = 1e9 / I.ME_EV


@pytest.fixture(scope="module")
def bks_tables():
    return O.tables(1e-3, 2.0, 40, 128)


class _Psi:
    """psi1, psi2, psi3 on a log grid of chi from the oracle's quadrature, cubic in ln chi."""

    def __init__(self, lo=1e-3, hi=2.0, n=60):
        self.lx = np.linspace(math.log(lo), math.log(hi), n)
        self.v = np.array([[O.psi(math.exp(x), k) for x in self.lx] for k in (1, 2, 3)])

    def __call__(self, chi):
        if chi <= math.exp(self.lx[0]):
            return np.zeros(3)  # below 1e-3 the radiative terms are ~1e-9 of the chi = 1 values
        x = math.log(chi)
        i = int(np.clip(np.searchsorted(self.lx, x) - 2, 0, len(self.lx) - 4))
        xs = self.lx[i:i + 4]
        w = [np.prod([(x - xs[m]) / (xs[l] - xs[m]) for m in range(4) if m != l]) for l in range(4)]
        return self.v[:, i:i + 4] @ np.array(w)


@pytest.fixture(scope="module")
def psi():
    return _Psi()


def _bfield(f, t):
    E, B = O.field_eval(f, np.zeros(3), t)
    return np.asarray(B)


def _bks(p0, S0, f, q, T, psi, dt=0.005):
    """RK4 of (p, S) with dp/dt = q (p/gamma) x B, dS/dt = Omega x S - Gamma[...] (E = 0)."""
    def rhs(t, y):
        p, S = y[:3], y[3:]
        B = _bfield(f, t)
        g = math.sqrt(1 + p @ p)
        v = p / g
        dp = q * np.cross(v, B)
        Om = -q * ((AE + 1 / g) * B - (AE * g / (g + 1)) * (v @ B) * v)
        dS = np.cross(Om, S)
        fv = np.cross(v, B)
        khat = p / math.sqrt(p @ p)
        fperp = fv - (fv @ khat) * khat
        nf = np.linalg.norm(fperp)
        if nf > 0:
            eps = -q * fperp / nf
            beta = np.cross(khat, eps)
            chi = ETA0 * math.sqrt(np.cross(p, B) @ np.cross(p, B))
            p1, p2, p3 = psi(chi)
            Gam = ALPHA / (math.sqrt(3) * math.pi * ETA0 * g)
            dS = dS - Gam * (p1 * S + p2 * (S @ khat) * khat - p3 * beta)
        return np.concatenate([dp, dS])

    y = np.concatenate([p0, S0]).astype(float)
    n = int(round(T / dt))
    out = {0: y[3:].copy()}
    for k in range(n):
        t = k * dt
        k1 = rhs(t, y)
        k2 = rhs(t + dt / 2, y + dt / 2 * k1)
        k3 = rhs(t + dt / 2, y + dt / 2 * k2)
        k4 = rhs(t + dt, y + dt * k3)
        y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        out[k + 1] = y[3:].copy()
    return out, dt


def _mc(b, f, flags, q, steps, dt, tables, seed, every):
    L = O.Particles.from_arrays(len(b["id"]), b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    L.init_tau(seed)
    out = {}
    for s in range(steps):
        O.lepton_step(tables, f, O.step_desc(dt, s * dt, s, seed, flags), q, L, None)
        if (s + 1) % every == 0:
            out[(s + 1) * dt] = L.view()["spin"].mean(axis=0)
    return out


def _at(ode, t):
    sol, h = ode
    return sol[int(round(t / h))]


FL = O.F_FULL & ~O.F_RECOIL


def test_bks_polarized_beam_in_constant_field(bks_tables, psi):
    """X7: SQA ensemble within 0.035 of the equation in every component at every sampled time (3 sigma of
    8000 spins is 0.02; the scheme's first-order bias in W dt = 0.03 adds ~0.01 along B, as in the
    Sokolov-Ternov pin); the beta-basis ensemble off by more than 0.3 in the transverse components (each
    emission projects them out, and by t = 2.5 nearly every electron has emitted), within 0.03 along B."""
    n, dt, steps = 8000, 0.025, 1200
    p = math.sqrt(GAMMA_1GEV ** 2 - 1)
    Bz = 1.0 / (ETA0 * p)  # chi = 1
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    b = I.lepton_beam(n, GAMMA_1GEV, direction=(1, 0, 0), spin="fixed", spin_dir=(1, 0, 0), seed=41)
    ode = _bks(b["mom"][0], np.array([1.0, 0, 0]), f, -1, steps * dt, psi)
    sqa = _mc(b, f, FL, -1, steps, dt, bks_tables, 41, 100)
    bet = _mc(b, f, FL | O.F_BETA_BASIS, -1, steps, dt, bks_tables, 41, 100)
    worst_sqa, worst_beta_t, worst_beta_z = 0.0, 0.0, 0.0
    for t, m in sqa.items():
        e = _at(ode, t)
        worst_sqa = max(worst_sqa, np.abs(m - e).max())
        mb = bet[t]
        worst_beta_t = max(worst_beta_t, np.abs(mb[:2] - e[:2]).max())
        worst_beta_z = max(worst_beta_z, abs(mb[2] - e[2]))
    assert worst_sqa < 0.035, worst_sqa
    assert worst_beta_t > 0.3, worst_beta_t
    assert worst_beta_z < 0.03, worst_beta_z
    # the equation's transverse polarization is still large at the end, so the test has power
    assert np.linalg.norm(_at(ode, steps * dt)[:2]) > 0.2


def test_bks_unpolarized_beam_in_rotating_field(bks_tables, psi):
    """X8: B of constant strength (chi = 1 while v is perpendicular to it) along z until t = 20, then
    turning to y within 2 pi x 3 ~ 19 (about a gyro-period); the SQA ensemble stays within 0.03 of the
    equation in every component before, during and after the turn; the beta-basis ensemble agrees
    before the turn and departs from the equation by more than 0.15 after it."""
    n, dt, steps = 12000, 0.025, 2400
    p = math.sqrt(GAMMA_1GEV ** 2 - 1)
    Bz = 1.0 / (ETA0 * p)
    f = O.field(O.FIELD_ROT_B, n_cycles=3.0, phase=-20.0, B0=(0, 0, Bz), eta0=ETA0)
    b = I.lepton_beam(n, GAMMA_1GEV, direction=(1, 0, 0), spin="random", seed=43)
    S0 = b["spin"].mean(axis=0)
    ode = _bks(b["mom"][0], S0, f, -1, steps * dt, psi)
    sqa = _mc(b, f, FL, -1, steps, dt, bks_tables, 43, 100)
    bet = _mc(b, f, FL | O.F_BETA_BASIS, -1, steps, dt, bks_tables, 43, 100)
    worst_sqa = max(np.abs(m - _at(ode, t)).max() for t, m in sqa.items())
    before = max(np.abs(m - _at(ode, t)).max() for t, m in bet.items() if t <= 20.0)
    after = max(np.abs(m - _at(ode, t)).max() for t, m in bet.items() if t >= 45.0)
    assert worst_sqa < 0.03, worst_sqa
    assert before < 0.03, before
    assert after > 0.15, after
    # the beam did polarize and the field did turn it
    assert _at(ode, 20.0)[2] < -0.3 and abs(_at(ode, steps * dt)[1]) > 0.1


def test_rotating_field_kind():
    """The field of the rotating-field test: |B| constant, along z before t = -phase, along y after
    t = -phase + 2 pi n_cycles, at angle (pi/2) u in between; E = 0."""
    f = O.field(O.FIELD_ROT_B, n_cycles=2.0, phase=-5.0, B0=(0, 0, 3.0), eta0=ETA0)
    for t, th in ((0.0, 0.0), (5.0, 0.0), (5.0 + 2 * math.pi, math.pi / 4), (5.0 + 4 * math.pi, math.pi / 2),
                  (100.0, math.pi / 2)):
        E, B = O.field_eval(f, np.array([1.0, -2.0, 3.0]), t)
        np.testing.assert_allclose(E, 0.0, atol=0)
        np.testing.assert_allclose(B, [0.0, 3.0 * math.sin(th), 3.0 * math.cos(th)], rtol=1e-15, atol=1e-15)


def test_beta_basis_emission_collapses_onto_beta(small_tables):
    """One emission step in a constant field: with the beta basis every emitter's spin ends at +-beta,
    and the fraction at -beta matches (w - g.beta)/(2w) averaged over the sampled photons (a mixture
    test: the mean of s_f.beta equals the mean of g.beta/w within statistics)."""
    n = 20000
    p = 3000.0
    Bz = 1.0 / (ETA0 * p)
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    b = I.lepton_beam(n, math.sqrt(p * p + 1), direction=(1, 0, 0), spin="random", seed=45)
    fl = (O.F_FULL & ~O.F_PUSH & ~O.F_TBMT) | O.F_BETA_BASIS
    L = O.Particles.from_arrays(n, b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=np.full(n, 1e-9))
    O.lepton_step(small_tables, f, O.step_desc(0.05, 0.0, 0, 5, fl), -1, L, None)
    s = L.view()["spin"]
    beta = np.array([0, 0, -1.0])  # electron along +x in B_z: eps = -y, beta = x cross eps = -z
    sb = s @ beta
    np.testing.assert_allclose(np.abs(sb), 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    # the expectation mode lands on the same mean along beta
    L2 = O.Particles.from_arrays(n, b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=np.full(n, 1e-9))
    O.lepton_step(small_tables, f, O.step_desc(0.05, 0.0, 0, 5, fl & ~O.F_SPIN_COLLAPSE), -1, L2, None)
    s2 = L2.view()["spin"]
    np.testing.assert_allclose(s2[:, :2], 0.0, atol=1e-15)
    assert sb.mean() == pytest.approx((s2 @ beta).mean(), abs=4.0 / math.sqrt(n))
