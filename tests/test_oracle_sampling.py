"""Pins of the oracle's sampling paths against the closed-form spectra of App. A, on the particles its
step functions actually emit (CPU only).

Every particle is loaded with an optical depth of zero, so each one converts (photon step) or emits
(lepton step) in its first step, and the distribution of the sampled energy fraction can be tested
against the spectrum written out from App. A with scipy's Bessel functions and a quadrature of this
module's own (nothing is taken from the oracle's tables or integrals):

* NBW (Sec. 5.2, Sec. 7.2): the positron fraction of pairs made by photons with xi3 = +1, -1, 0 at
  chi_gamma = 0.5, 1, 10, 99 follows w0(lambda; xi3) = IntK13(u~') + rho K23(u~') - xi3 K23(u~').
  This pins the folded ICDF, orc_nbw_mu and the side choice of the photon step.
* NLC (Sec. 5.1, Sec. 7.1): the photon fraction emitted by leptons with s.beta = +1, -1, 0 at
  chi = 0.1, 1, 10, 99 follows w(lambda; s.beta) = -IntK13(u') + kappa K23(u') + lambda s.beta K13(u'),
  and for unpolarized leptons the photons with xi3 = +1 and xi3 = -1 follow (w + K23)/2 and (w - K23)/2
  (App. A.1: the unpolarized F0 = w, F3 = K23; their split as in Sec. 7.1).
* The per-step probability decision (Sec. 4.1, 5.1, 5.2: event if r1 < W dt, branch by the same r1):
  event frequency W dt within binomial statistics, with W from the closed-form rate, and the sampled
  spectrum the spin (polarization) mixture, so the branch share W_down (1 - s.beta) / (2 W_s) holds.
* The oracle's mixture-quantile mode (the learned sampler's target on the step): its fractions follow
  the same w(lambda; s.beta), and each inverts the exact mixture CDF at the lepton's own r2.
* T-BMT (Sec. 8.3): in a Wien filter (E = v B, E perpendicular to B and v) the momentum is constant and
  the spin precesses about B at (1 + a) B / gamma^2 (the textbook Wien-filter rotation) in the standard
  form; the form as printed gives (a + 1/gamma) B / gamma^2.

Each statistical test also checks its own power where a plausible mistake would change the
distribution: the wrong spectrum (swapped sign of xi3 or s.beta, a fold that keeps one side) must be
rejected by the same statistic.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2511_08929_gb300 import inputs as I

sp = pytest.importorskip("scipy.special")
st = pytest.importorskip("scipy.stats")

ALPHA = 7.2973525693e-3
AE = ALPHA / (2 * math.pi)
ETA0 = I.eta0_for_wavelength(0.8)
N = 20000
P_MIN = 1e-3  # a KS p-value below this fails a test (each test makes a few comparisons)


# ------------------------------------------------------------------------------------------
# closed-form spectra (App. A) with scipy's K_nu and this module's own quadrature
# ------------------------------------------------------------------------------------------
_GX, _GW = np.polynomial.legendre.leggauss(10)


def _intk13_table():
    """int_x^inf K_{1/3}(t) dt on a log grid of x: panel sums of Gauss-Legendre quadrature in ln t,
    accumulated from the top (the integrand is negligible beyond t = 400)."""
    lx = np.linspace(math.log(1e-14), math.log(400.0), 6001)
    a, b = lx[:-1], lx[1:]
    m, r = 0.5 * (a + b), 0.5 * (b - a)
    t = m[:, None] + r[:, None] * _GX[None, :]
    seg = (np.exp(t) * sp.kv(1.0 / 3.0, np.exp(t)) * _GW[None, :]).sum(1) * r
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [1e-300]])
    return lx, np.log(np.maximum(tail, 1e-300))


_LX, _LTAIL = _intk13_table()
_C0 = math.gamma(1.0 / 3.0) / 2.0 * 2.0 ** (1.0 / 3.0) * 1.5  # int_0^x K13 ~ C0 x^{2/3} as x -> 0


def intk13(x):
    x = np.asarray(x, dtype=np.float64)
    big = np.exp(np.interp(np.log(np.clip(x, 1e-14, 400.0)), _LX, _LTAIL))
    big = np.where(x >= 400.0, 0.0, big)
    return np.where(x < 1e-14, math.pi / math.sqrt(3.0) - _C0 * np.cbrt(x * x), big)


def nlc_density(lam, chi, sbeta=0.0, xi3_sign=0):
    """w(lambda; s.beta) per unit lambda (App. A.1); xi3_sign = +1 / -1: the part (w +- K23)/2 carried by
    photons with xi3 = +1 / -1 (unpolarized leptons only)."""
    lam = np.asarray(lam, dtype=np.float64)
    up = 2.0 * lam / (3.0 * chi * (1.0 - lam))
    k13, k23, ik = sp.kv(1.0 / 3.0, up), sp.kv(2.0 / 3.0, up), intk13(up)
    kappa = 1.0 / (1.0 - lam) + (1.0 - lam)
    w = -ik + kappa * k23 + sbeta * lam * k13
    if xi3_sign:
        w = 0.5 * (w + xi3_sign * k23)
    return w


def nbw_density(lam, chi, xi3):
    """w0(lambda; xi3) per unit positron fraction lambda (App. A.2)."""
    lam = np.asarray(lam, dtype=np.float64)
    ut = 2.0 / (3.0 * chi * lam * (1.0 - lam))
    k23, ik = sp.kv(2.0 / 3.0, ut), intk13(ut)
    rho = (1.0 - lam) / lam + lam / (1.0 - lam)
    return ik + rho * k23 - xi3 * k23


class Spectrum:
    """Normalised CDF of a density on (0, 1) by composite Gauss-Legendre quadrature on a grid that is
    fine near both ends.  NLC densities are integrated in v = lambda^{1/3} (the lambda^{-2/3} infrared
    behaviour becomes a finite integrand)."""

    def __init__(self, density, cube=False):
        if cube:
            g = np.concatenate([np.linspace(0.0, 0.9, 3001), 1.0 - np.logspace(-1, -9, 3001)[1:]])
            to_lam = lambda v: v ** 3
            jac = lambda v: 3.0 * v * v
        else:
            g = np.concatenate([np.logspace(-14, -2, 1200)[:-1], np.linspace(0.01, 0.99, 4001),
                                1.0 - np.logspace(-2, -14, 1200)[1:]])
            g = np.concatenate([[0.0], g, [1.0]])
            to_lam = lambda v: v
            jac = lambda v: np.ones_like(v)
        a, b = g[:-1], g[1:]
        m, r = 0.5 * (a + b), 0.5 * (b - a)
        v = m[:, None] + r[:, None] * _GX[None, :]
        lam = np.clip(to_lam(v), 1e-300, 1.0 - 1e-16)
        with np.errstate(all="ignore"):
            f = np.nan_to_num(density(lam) * jac(v), nan=0.0, posinf=0.0)
        seg = (f * _GW[None, :]).sum(1) * r
        self.total = seg.sum()
        self.grid = g
        self.cum = np.concatenate([[0.0], np.cumsum(seg)]) / self.total
        self.cube = cube

    def cdf(self, lam):
        v = np.cbrt(lam) if self.cube else np.asarray(lam)
        return np.interp(v, self.grid, self.cum)

    def total_lambda(self):
        """int_0^1 density d lambda (the rate integral)."""
        return self.total


def ks_p(samples, spec):
    return st.kstest(np.asarray(samples), spec.cdf).pvalue


@pytest.fixture(scope="module")
def tb():
    """Oracle tables over the chi range of these tests."""
    return O.tables(0.05, 200.0, 64, 128)


# ------------------------------------------------------------------------------------------
# beams in a constant magnetic field: particles along +x, B along z
#   leptons (electron convention, q = -1): eps = -y, beta = k x eps = -z   (reading C9)
#   photons: eps = -y, beta = -z
# ------------------------------------------------------------------------------------------
EPS = np.array([0.0, -1.0, 0.0])
BETA = np.array([0.0, 0.0, -1.0])
KHAT = np.array([1.0, 0.0, 0.0])


def _photons(chi, P, energy=2000.0, n=N, seed=3):
    b = I.photon_beam(n, energy, direction=(1, 0, 0), P=P, seed=seed)
    G = O.Particles.from_arrays(n, b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=np.zeros(n))
    f = O.field(O.FIELD_CONST, B0=(0, 0, chi / (ETA0 * energy)), eta0=ETA0)
    return G, f


def _electrons(chi, spin, gamma=2000.0, n=N, seed=4, tau=0.0):
    b = I.lepton_beam(n, gamma, direction=(1, 0, 0), spin="fixed" if np.linalg.norm(spin) > 0 else "zero",
                      spin_dir=spin if np.linalg.norm(spin) > 0 else (0, 0, 1), seed=seed)
    b["spin"] = np.tile(np.asarray(spin, dtype=np.float64), (n, 1))
    L = O.Particles.from_arrays(n, b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=np.full(n, tau))
    pm = math.sqrt(gamma * gamma - 1.0)
    f = O.field(O.FIELD_CONST, B0=(0, 0, chi / (ETA0 * pm)), eta0=ETA0)
    return L, f, pm


# ------------------------------------------------------------------------------------------
# NBW: positron fractions of the created pairs (Sec. 5.2, Sec. 7.2)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("chi", [0.5, 1.0, 10.0, 99.0])
def test_nbw_positron_fraction_follows_w0(chi, tb):
    energy = 2000.0
    for xi3, P in ((1.0, (0.0, 1.0, 0.0)), (-1.0, (0.0, 0.0, 1.0)), (0.0, (1.0, 0.0, 0.0))):
        # P along eps: xi3 = +1; along beta: xi3 = -1; along k: circular, xi3 = 0
        G, f = _photons(chi, P, energy)
        el, po = O.Particles(N), O.Particles(N)
        ctr = O.photon_step(tb, f, O.step_desc(0.01, 0.0, 0, 11, O.F_FULL & ~O.F_MOVE), G, el, po)
        assert ctr.events == N and el.n == po.n == N and G.n == 0
        e, p = el.view(), po.view()
        np.testing.assert_allclose(e["mom"] + p["mom"], np.tile([energy, 0, 0], (N, 1)), rtol=1e-13, atol=1e-9)
        lam = p["mom"][:, 0] / energy
        spec = Spectrum(lambda l: nbw_density(l, chi, xi3))
        assert ks_p(lam, spec) > P_MIN, (chi, xi3)
        # both sides of lambda = 1/2 are populated evenly (w0 is symmetric under lambda <-> 1 - lambda)
        assert abs((lam < 0.5).mean() - 0.5) < 4 * math.sqrt(0.25 / N)
        # power: a fold that always returned the lambda <= 1/2 side is rejected at once
        assert ks_p(np.minimum(lam, 1 - lam), spec) < 1e-12
        if xi3 != 0.0 and chi <= 1.0:
            # where the xi3 = +-1 spectra differ in shape the test tells them apart
            assert ks_p(lam, Spectrum(lambda l: nbw_density(l, chi, -xi3))) < 1e-4


def test_nbw_fraction_grid_of_the_fold(tb):
    """orc_nbw_mu inverts mu (1 - mu) = 2 / (3 chi u~') on mu <= 1/2 (the folded variable x = u~' - 8/(3 chi)
    measured from the centre lambda = 1/2): mu = 1/2 at x = 0, and u~' recomputed from mu gives x back."""
    for chi in (0.5, 3.0, 99.0):
        assert O.nbw_mu(chi, 0.0) == pytest.approx(0.5, abs=1e-8)
        for x in (1e-6, 0.3, 5.0, 300.0):
            mu = O.nbw_mu(chi, x)
            assert 0.0 < mu < 0.5
            assert 2.0 / (3.0 * chi * mu * (1.0 - mu)) - 8.0 / (3.0 * chi) == pytest.approx(x, rel=1e-9)


# ------------------------------------------------------------------------------------------
# NLC: energy fractions of the emitted photons (Sec. 5.1, Sec. 7.1)
# ------------------------------------------------------------------------------------------
FL_EMIT = O.F_FULL & ~O.F_PUSH & ~O.F_TBMT & ~O.F_MOVE


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0, 99.0])
def test_nlc_photon_fraction_follows_w(chi, tb):
    for sbeta in (1.0, -1.0):
        L, f, pm = _electrons(chi, sbeta * BETA)
        G = O.Particles(N)
        ctr = O.lepton_step(tb, f, O.step_desc(0.01, 0.0, 0, 12, FL_EMIT), -1, L, G)
        assert ctr.events == N and G.n == N
        g = G.view()
        lam = g["mom"][:, 0] / pm
        np.testing.assert_allclose(g["mom"][:, 1:], 0.0, atol=1e-9)
        spec = Spectrum(lambda l: nlc_density(l, chi, sbeta), cube=True)
        assert ks_p(lam, spec) > P_MIN, (chi, sbeta)
        if chi >= 1.0:
            # the opposite spin's spectrum is rejected: the s.beta term of w is resolved
            assert ks_p(lam, Spectrum(lambda l: nlc_density(l, chi, -sbeta), cube=True)) < 1e-6


@pytest.mark.parametrize("chi,sbeta", [(1.0, 0.6), (10.0, -0.8)])
def test_mixture_quantile_mode(chi, sbeta, tb):
    """The oracle mode F_MIX_QUANTILE (the learned sampler's target on the step, Sec. 5.1): every
    emission's u' is the exact quantile of the mixture w(lambda; s.beta) at the lepton's own r2, so the
    oracle's mixture CDF there returns r2 (1e-9), and the fractions follow the closed-form w(lambda; s.beta)
    (KS); with the sign of s.beta flipped the CDF misses r2 by more than 1e-3."""
    n = 1500
    L, f, pm = _electrons(chi, sbeta * BETA, n=n, seed=9)
    G = O.Particles(n)
    ctr = O.lepton_step(tb, f, O.step_desc(0.01, 0.0, 0, 13, FL_EMIT | O.F_MIX_QUANTILE), -1, L, G)
    assert ctr.events == n and G.n == n
    g, l = G.view(), L.view()
    lam = g["mom"][:, 0] / pm
    assert ks_p(lam, Spectrum(lambda x: nlc_density(x, chi, sbeta), cube=True)) > P_MIN
    parent = {O.child_ids(int(i), 13, 0)[0]: k for k, i in enumerate(l["id"])}
    worst, worst_flip = 0.0, 0.0
    for m in range(0, n, 15):
        k = parent[int(g["id"][m])]
        lm = g["mom"][m, 0] / (g["mom"][m, 0] + l["mom"][k, 0])
        ln_up = math.log(2.0 * lm / (3.0 * chi * (1.0 - lm)))
        r2 = O.uniform_pair(int(l["id"][k]), 13, 0, 1)[0]
        worst = max(worst, abs(O.mlp_cdf(chi, sbeta, ln_up) - r2))
        worst_flip = max(worst_flip, abs(O.mlp_cdf(chi, -sbeta, ln_up) - r2))
    assert worst < 1e-9, worst
    assert worst_flip > 1e-3, worst_flip


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0, 99.0])
def test_nlc_unpolarized_split_by_xi3(chi, tb):
    """Unpolarized leptons (s = 0): photons come out with xi3 = +-1 exactly (App. A.1: with s_i = 0 the
    collapsed s_f is +-beta, F1 = F2 = 0), and those with xi3 = +1 / -1 follow (w + K23)/2 / (w - K23)/2;
    their numbers split as int (w +- K23) / int 2 w (Sec. 7.1)."""
    L, f, pm = _electrons(chi, (0.0, 0.0, 0.0), seed=5)
    G = O.Particles(N)
    O.lepton_step(tb, f, O.step_desc(0.01, 0.0, 0, 13, FL_EMIT), -1, L, G)
    g = G.view()
    lam = g["mom"][:, 0] / pm
    xi = np.array([O.P_to_stokes(P, EPS, BETA, KHAT) for P in g["spin"]])
    np.testing.assert_allclose(np.abs(xi[:, 2]), 1.0, atol=1e-12)
    np.testing.assert_allclose(xi[:, :2], 0.0, atol=1e-12)
    plus = xi[:, 2] > 0
    sp_all = Spectrum(lambda l: nlc_density(l, chi), cube=True)
    assert ks_p(lam, sp_all) > P_MIN
    s_plus = Spectrum(lambda l: nlc_density(l, chi, xi3_sign=1), cube=True)
    s_minus = Spectrum(lambda l: nlc_density(l, chi, xi3_sign=-1), cube=True)
    assert ks_p(lam[plus], s_plus) > P_MIN and ks_p(lam[~plus], s_minus) > P_MIN
    frac = s_plus.total_lambda() / sp_all.total_lambda()
    assert abs(plus.mean() - frac) < 4 * math.sqrt(frac * (1 - frac) / N), (plus.mean(), frac)
    # power: the two subsets' spectra are told apart where they differ in shape
    if chi <= 1.0:
        assert ks_p(lam[plus], s_minus) < 1e-6


# ------------------------------------------------------------------------------------------
# per-step probability decision (QED_F_TAU off): frequency and branch share
# ------------------------------------------------------------------------------------------
PREF_NLC = ALPHA / (math.sqrt(3.0) * math.pi * ETA0)


@pytest.mark.parametrize("sbeta", [1.0, 0.3, -1.0])
def test_probability_mode_lepton_frequency_and_branch(sbeta, tb):
    chi, gamma = 4.0, 2000.0
    n = 40000
    s_up = Spectrum(lambda l: nlc_density(l, chi, 1.0), cube=True).total_lambda()
    s_dn = Spectrum(lambda l: nlc_density(l, chi, -1.0), cube=True).total_lambda()
    W_up, W_dn = PREF_NLC / gamma * s_up, PREF_NLC / gamma * s_dn
    Ws = W_up * (1 + sbeta) / 2 + W_dn * (1 - sbeta) / 2
    dt = 0.3 / Ws  # event probability 0.3 per step
    L, f, pm = _electrons(chi, sbeta * BETA, gamma=gamma, n=n, seed=6, tau=1.0)
    G = O.Particles(n)
    ctr = O.lepton_step(tb, f, O.step_desc(dt, 0.0, 0, 14, FL_EMIT & ~O.F_TAU), -1, L, G)
    p = Ws * dt
    assert abs(ctr.events / n - p) < 4 * math.sqrt(p * (1 - p) / n), (ctr.events / n, p)
    lam = G.view()["mom"][:, 0] / pm
    assert ks_p(lam, Spectrum(lambda l: nlc_density(l, chi, sbeta), cube=True)) > P_MIN
    if abs(sbeta) == 1.0:
        assert ks_p(lam, Spectrum(lambda l: nlc_density(l, chi, -sbeta), cube=True)) < 1e-6


@pytest.mark.parametrize("xi3,P", [(1.0, (0.0, 1.0, 0.0)), (-1.0, (0.0, 0.0, 1.0))])
def test_probability_mode_photon_frequency_and_branch(xi3, P, tb):
    chi, energy = 1.0, 2000.0
    n = 40000
    J = Spectrum(lambda l: nbw_density(l, chi, xi3)).total_lambda()
    W = ALPHA / (math.sqrt(3.0) * math.pi * ETA0 * energy) * J
    dt = 0.3 / W
    G, f = _photons(chi, P, energy, n=n, seed=7)
    G.a["tau"][:n] = 1.0
    el, po = O.Particles(n), O.Particles(n)
    ctr = O.photon_step(tb, f, O.step_desc(dt, 0.0, 0, 15, O.F_FULL & ~O.F_MOVE & ~O.F_TAU), G, el, po)
    p = W * dt
    assert abs(ctr.events / n - p) < 4 * math.sqrt(p * (1 - p) / n), (ctr.events / n, p)
    lam = po.view()["mom"][:, 0] / energy
    assert ks_p(lam, Spectrum(lambda l: nbw_density(l, chi, xi3))) > P_MIN


# ------------------------------------------------------------------------------------------
# table-free rejection sampling (Sec. 4.2, the f = r^3 proposal): frequency and spectrum
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("sbeta", [1.0, -0.4])
def test_rejection_lepton_frequency_and_spectrum(sbeta, tb):
    """Candidates lambda = r1^3 accepted with probability 3 r1^2 (dW/dlambda) dt: the event frequency is
    W_s dt and the accepted fractions follow w(lambda; s.beta), with no table involved in either."""
    chi, gamma = 4.0, 2000.0
    n = 100000
    s_up = Spectrum(lambda l: nlc_density(l, chi, 1.0), cube=True).total_lambda()
    s_dn = Spectrum(lambda l: nlc_density(l, chi, -1.0), cube=True).total_lambda()
    Ws = PREF_NLC / gamma * (s_up * (1 + sbeta) / 2 + s_dn * (1 - sbeta) / 2)
    dt = 0.05 / Ws
    L, f, pm = _electrons(chi, sbeta * BETA, gamma=gamma, n=n, seed=8, tau=1.0)
    G = O.Particles(n)
    ctr = O.lepton_step(tb, f, O.step_desc(dt, 0.0, 0, 16, (FL_EMIT & ~O.F_TAU) | O.F_REJECT), -1, L, G)
    assert ctr.bound_exceeded == 0
    p = Ws * dt
    assert abs(ctr.events / n - p) < 4 * math.sqrt(p * (1 - p) / n), (ctr.events / n, p)
    lam = G.view()["mom"][:, 0] / pm
    assert ks_p(lam, Spectrum(lambda l: nlc_density(l, chi, sbeta), cube=True)) > P_MIN
    if sbeta == 1.0:
        assert ks_p(lam, Spectrum(lambda l: nlc_density(l, chi, -1.0), cube=True)) < 1e-6
    assert np.all(L.view()["tau"] == 1.0)  # no optical depth in this mode


@pytest.mark.parametrize("xi3,P", [(1.0, (0.0, 1.0, 0.0)), (-1.0, (0.0, 0.0, 1.0))])
def test_rejection_photon_frequency_and_spectrum(xi3, P, tb):
    """Candidate positron fractions lambda = r1 accepted with probability (dW/dlambda) dt."""
    chi, energy = 1.0, 2000.0
    n = 100000
    J = Spectrum(lambda l: nbw_density(l, chi, xi3)).total_lambda()
    W = ALPHA / (math.sqrt(3.0) * math.pi * ETA0 * energy) * J
    dt = 0.05 / W
    G, f = _photons(chi, P, energy, n=n, seed=9)
    G.a["tau"][:n] = 1.0
    el, po = O.Particles(n), O.Particles(n)
    ctr = O.photon_step(tb, f, O.step_desc(dt, 0.0, 0, 17, (O.F_FULL & ~O.F_MOVE & ~O.F_TAU) | O.F_REJECT), G, el, po)
    assert ctr.bound_exceeded == 0
    p = W * dt
    assert abs(ctr.events / n - p) < 4 * math.sqrt(p * (1 - p) / n), (ctr.events / n, p)
    lam = po.view()["mom"][:, 0] / energy
    assert ks_p(lam, Spectrum(lambda l: nbw_density(l, chi, xi3))) > P_MIN


def test_rejection_bound_is_counted(tb):
    """A step so long that 3 r^2 (dW/dlambda) dt exceeds 1 for some candidates is counted (the method's
    requirement, Sec. 4.2); then the accepted spectrum is distorted, which the counter reports."""
    chi, gamma = 4.0, 2000.0
    L, f, pm = _electrons(chi, BETA, gamma=gamma, n=20000, seed=10, tau=1.0)
    dt = 5.0 / (PREF_NLC / gamma)
    ctr = O.lepton_step(tb, f, O.step_desc(dt, 0.0, 0, 18, (FL_EMIT & ~O.F_TAU) | O.F_REJECT), -1, L, None)
    assert ctr.bound_exceeded > 0


# ------------------------------------------------------------------------------------------
# T-BMT in a Wien filter (Sec. 8.3): both forms against their closed forms
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("q", [-1, 1])
def test_tbmt_wien_filter_precession(q, tb):
    gamma, Bz, dt, n = 3.0, 0.5, 0.01, 300
    pm = math.sqrt(gamma * gamma - 1.0)
    v = pm / gamma
    b = {"pos": np.zeros((1, 3)), "mom": np.array([[pm, 0.0, 0.0]]), "spin": np.array([[1.0, 0.0, 0.0]]),
         "w": np.ones(1), "id": np.array([9], dtype=np.uint64)}
    # E = v B along y: the Lorentz force q (E + v x B) vanishes
    f = O.field(O.FIELD_CONST, E0=(0.0, v * Bz, 0.0), B0=(0.0, 0.0, Bz), eta0=ETA0)
    L = O.Particles.from_arrays(1, b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    Lp = O.Particles.from_arrays(1, b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    for s in range(n):
        O.lepton_step(tb, f, O.step_desc(dt, s * dt, s, 1, O.F_TBMT | O.F_MOVE), q, L, None)
        O.lepton_step(tb, f, O.step_desc(dt, s * dt, s, 1, O.F_TBMT | O.F_TBMT_PAPER | O.F_MOVE), q, Lp, None)
    # Omega = -q (rate) B z: the spin turns by -q rate B n dt about z
    for P, rate in ((L, (1.0 + AE) / gamma ** 2), (Lp, (AE + 1.0 / gamma) / gamma ** 2)):
        s_ = P.view()["spin"][0]
        ang = math.atan2(s_[1], s_[0])
        assert ang == pytest.approx(-q * rate * Bz * n * dt, abs=1e-12)
        assert s_[2] == pytest.approx(0.0, abs=1e-15) and np.linalg.norm(s_) == pytest.approx(1.0, abs=1e-14)
    # the two forms differ by (1 - 1/gamma) B / gamma^2: here a factor of ~3 in the angle
    a1 = math.atan2(L.view()["spin"][0][1], L.view()["spin"][0][0])
    a2 = math.atan2(Lp.view()["spin"][0][1], Lp.view()["spin"][0][0])
    assert abs(a1) > 2.5 * abs(a2)
