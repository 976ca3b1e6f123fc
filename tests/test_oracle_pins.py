"""Pins of the FP64 oracle to things other than itself: published test vectors, an independent
special-function library (scipy), closed forms and limits the paper or the mathematics fixes,
and algebraic invariants of the spectra.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle as O

sp = pytest.importorskip("scipy.special")
si = pytest.importorskip("scipy.integrate")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = 7.2973525693e-3


# ------------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# ------------------------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert O.philox4x32_10(v[0:4], v[4:6]) == v[6:10]
        n += 1
    assert n == 3


def test_uniform_open_interval_and_exactness():
    L = O.lib()
    assert L.orc_uniform(0, 0) == 0.5 * 2.0 ** -52
    assert L.orc_uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert 0.0 < L.orc_uniform(0xFFFFFFFF, 0xFFFFFFFF) < 1.0
    # low 12 bits of the high word are discarded; everything else changes the value
    assert L.orc_uniform(0x00000FFF, 7) == L.orc_uniform(0, 7)
    assert L.orc_uniform(0x00001000, 7) != L.orc_uniform(0, 7)


def test_draws_are_keyed_by_id_step_slot():
    a = O.uniform_pair(5, 1, 10, 0)
    assert a == O.uniform_pair(5, 1, 10, 0)
    assert a != O.uniform_pair(6, 1, 10, 0)
    assert a != O.uniform_pair(5, 1, 11, 0)
    assert a != O.uniform_pair(5, 1, 10, 1)
    assert a != O.uniform_pair(5, 2, 10, 0)
    # birth optical depth is an exponential(1) variate: mean 1, variance 1
    taus = np.array([O.birth_tau(i, 9) for i in range(20000)])
    assert abs(taus.mean() - 1.0) < 0.03 and abs(taus.var() - 1.0) < 0.06


# ------------------------------------------------------------------------------------------
# Bessel functions: against scipy and DLMF identities
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("x", [1e-12, 1e-8, 1e-4, 1e-2, 0.1, 0.7, 1.0, 3.0, 10.0, 50.0, 300.0])
def test_bessel_against_scipy(x):
    k13, k23, ik = O.bessel(x)
    assert k13 == pytest.approx(sp.kv(1.0 / 3.0, x), rel=2e-14)
    assert k23 == pytest.approx(sp.kv(2.0 / 3.0, x), rel=2e-14)
    if x < 0.1:
        # int_x^inf = pi/sqrt3 - int_0^x (DLMF 10.43.19); quad on the short interval is accurate
        ref = math.pi / math.sqrt(3.0) - si.quad(lambda y: sp.kv(1.0 / 3.0, y), 0, x, epsabs=0, epsrel=1e-13,
                                                  limit=200)[0]
        assert ik == pytest.approx(ref, rel=1e-12)
    else:
        ref = si.quad(lambda y: sp.kve(1.0 / 3.0, y) * math.exp(x - y), x, np.inf, epsabs=0, epsrel=1e-13,
                      limit=500)[0]
        assert ik * math.exp(x) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("x", [1e3, 3e4])
def test_bessel_scaled_large_argument(x):
    s13, s23, sik = O.bessel(x, scaled=True)
    assert s13 == pytest.approx(sp.kve(1.0 / 3.0, x), rel=2e-14)
    assert s23 == pytest.approx(sp.kve(2.0 / 3.0, x), rel=2e-14)
    # int_x^inf K_nu ~ K_nu(x) (1 - (1/2)/x + ...) for large x: the ratio tends to 1 from below
    assert 1.0 - 1.0 / x < sik / s13 < 1.0


def test_bessel_identities():
    # int_0^inf K_nu = pi / (2 cos(nu pi / 2))  (DLMF 10.43.19): IntK13(0) = pi/sqrt(3)
    assert O.bessel(1e-14)[2] == pytest.approx(math.pi / math.sqrt(3.0), rel=1e-8)
    for x in [0.05, 0.5, 2.0, 8.0]:
        k13, k23, ik = O.bessel(x)
        # recurrence K_{5/3} = K_{1/3} + (4/(3x)) K_{2/3}  (DLMF 10.29.1)
        assert k13 + 4.0 / (3.0 * x) * k23 == pytest.approx(sp.kv(5.0 / 3.0, x), rel=1e-13)
        # d/dx IntK13 = -K13 (central difference)
        h = 1e-5 * x
        d = (O.bessel(x + h)[2] - O.bessel(x - h)[2]) / (2 * h)
        assert d == pytest.approx(-k13, rel=1e-8)
    # int_0^inf K_{2/3} = pi (DLMF 10.43.19 with nu = 2/3), using the oracle's K23
    tot = si.quad(lambda t: O.bessel(t ** 3)[1] * 3 * t * t, 0, 4.0, epsabs=0, epsrel=1e-11, limit=200)[0]
    assert tot == pytest.approx(math.pi, rel=1e-9)


# ------------------------------------------------------------------------------------------
# Spectra (App. A): algebraic structure
# ------------------------------------------------------------------------------------------
def _rh_basis(seed):
    rng = np.random.default_rng(seed)
    k = rng.normal(size=3)
    k /= np.linalg.norm(k)
    e = rng.normal(size=3)
    e -= e.dot(k) * k
    e /= np.linalg.norm(e)
    return e, np.cross(k, e), k


def _unit(rng, n=1):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _sph(a):
    return np.array([math.sin(a[0]) * math.cos(a[1]), math.sin(a[0]) * math.sin(a[1]), math.cos(a[0])])


def test_nlc_unpolarized_limit():
    """s_i = s_f = 0: F = (-IntK13 + kappa K23) + xi3 K23 (Eq. F^unpol) and <xi3> = K23/(...)."""
    eps, beta, k = _rh_basis(1)
    for chi, lam in [(0.1, 0.2), (1.0, 0.5), (10.0, 0.9)]:
        up = 2 * lam / (1 - lam) / (3 * chi)
        b = O.bessel(up)
        F = O.nlc_stokes(lam, b, np.zeros(3), np.zeros(3), eps, beta, k)
        kap = 1 / (1 - lam) + (1 - lam)
        assert F[0] == pytest.approx(-b[2] + kap * b[1], rel=1e-14)
        assert F[1] == 0 and F[2] == 0
        assert F[3] == pytest.approx(b[1], rel=1e-14)


def _min_margin_nlc(chi, lam, eps, beta, k, left_handed=False, starts=12, seed=0):
    from scipy.optimize import minimize
    up = 2 * lam / (1 - lam) / (3 * chi)
    b = O.bessel(up, scaled=True)
    bb = -beta if left_handed else beta

    def f(a):
        si_, sf_ = _sph(a[0:2]), _sph(a[2:4])
        F = O.nlc_stokes(lam, b, si_, sf_, eps, bb, k)
        return (F[0] - np.linalg.norm(F[1:])) / F[0]

    rng = np.random.default_rng(seed)
    best = 1e9
    for _ in range(starts):
        r = minimize(f, rng.uniform(0, 2 * math.pi, 4), method="Nelder-Mead",
                     options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 4000})
        best = min(best, r.fun)
    return best


@pytest.mark.parametrize("chi,lam", [(0.1, 0.05), (0.1, 0.8), (1.0, 0.3), (10.0, 0.7), (100.0, 0.95)])
def test_nlc_positivity_and_completeness_right_handed(chi, lam):
    """For pure initial/final spins and photon states the probability F0 - |F| is >= 0 and reaches 0:
    with beta = k x eps the printed F0..F3 form a valid (complete, positive) density."""
    eps, beta, k = _rh_basis(2)
    m = _min_margin_nlc(chi, lam, eps, beta, k)
    assert m > -1e-10
    assert m < 1e-6


def test_nlc_left_handed_basis_breaks_positivity():
    """The basis reading is pinned: with k x beta = eps (left-handed) the same formulas go negative."""
    eps, beta, k = _rh_basis(3)
    assert _min_margin_nlc(0.1, 0.8, eps, beta, k, left_handed=True) < -0.1


def _G_printed(lam, b, spv, sev, eps, beta, k):
    """G with the last G3 term as printed in the Bessel form (sign opposite to the Airy form)."""
    G = O.nbw_G(lam, b, spv, sev, eps, beta, k)
    rho = (1 - lam) / lam + lam / (1 - lam)
    G[3] -= 2 * (1 - rho / 2) * b[1] * spv.dot(k) * sev.dot(k)
    return G


def _min_margin_nbw(chi, lam, eps, beta, k, printed=False, starts=12, seed=0):
    from scipy.optimize import minimize
    ut = 2 * (1 / lam + 1 / (1 - lam)) / (3 * chi)
    b = O.bessel(ut, scaled=True)
    fn = _G_printed if printed else O.nbw_G

    def f(a):
        G = fn(lam, b, _sph(a[0:2]), _sph(a[2:4]), eps, beta, k)
        return (G[0] - np.linalg.norm(G[1:])) / G[0]

    rng = np.random.default_rng(seed)
    best = 1e9
    for _ in range(starts):
        r = minimize(f, rng.uniform(0, 2 * math.pi, 4), method="Nelder-Mead",
                     options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 4000})
        best = min(best, r.fun)
    return best


@pytest.mark.parametrize("chi,lam", [(0.5, 0.5), (1.0, 0.3), (10.0, 0.05), (100.0, 0.7)])
def test_nbw_positivity_and_completeness(chi, lam):
    eps, beta, k = _rh_basis(4)
    m = _min_margin_nbw(chi, lam, eps, beta, k)
    assert m > -1e-10
    assert m < 1e-6


def test_nbw_printed_G3_sign_breaks_positivity():
    """The G3 sign reading is pinned: the printed Bessel-form sign yields negative probabilities."""
    eps, beta, k = _rh_basis(5)
    assert _min_margin_nbw(1.0, 0.3, eps, beta, k, printed=True) < -0.05


def test_nbw_marginals_match_j_and_four_states_sum():
    rng = np.random.default_rng(6)
    eps, beta, k = _rh_basis(6)
    for chi, lam in [(0.7, 0.2), (5.0, 0.6), (50.0, 0.95)]:
        ut = 2 * (1 / lam + 1 / (1 - lam)) / (3 * chi)
        b = O.bessel(ut, scaled=True)
        xi = _unit(rng)[0] * rng.uniform(0.2, 1.0)
        w0, je, jp = O.nbw_j(lam, b, xi, eps, beta, k)

        def Gf(spv, sev):
            G = O.nbw_G(lam, b, spv, sev, eps, beta, k)
            return G[0] + xi.dot(G[1:])

        se, spv = _unit(rng)[0], _unit(rng)[0]
        # averaging over the positron spin leaves w0 + s_e . j_e (Eq. for <s_e>), and vice versa
        assert 0.5 * (Gf(spv, se) + Gf(-spv, se)) == pytest.approx(w0 + se.dot(je), rel=1e-13)
        assert 0.5 * (Gf(spv, se) + Gf(spv, -se)) == pytest.approx(w0 + spv.dot(jp), rel=1e-13)
        Se, Sp = je / np.linalg.norm(je), jp / np.linalg.norm(jp)
        tot = sum(Gf(a * Sp, c * Se) for a in (-1, 1) for c in (-1, 1))
        assert tot == pytest.approx(4 * w0, rel=1e-13)
        # xi = 0: the electron's mean spin is (1/(1-lambda)) K13 beta / w0
        w00, je0, _ = O.nbw_j(lam, b, np.zeros(3), eps, beta, k)
        np.testing.assert_allclose(je0, b[0] / (1 - lam) * beta, rtol=1e-14, atol=1e-300)


def test_nlc_final_spin_marginal():
    """Summing F0 over s_f = +-S_SQA gives 2w; the SQA collapse reproduces <s_f> = g/w in mean."""
    rng = np.random.default_rng(7)
    eps, beta, k = _rh_basis(7)
    for chi, lam in [(0.1, 0.1), (2.0, 0.5)]:
        up = 2 * lam / (1 - lam) / (3 * chi)
        b = O.bessel(up, scaled=True)
        s = _unit(rng)[0] * 0.9
        w, g = O.nlc_wg(lam, b, s, eps, beta, k)
        S = g / np.linalg.norm(g)
        Fp = O.nlc_stokes(lam, b, s, S, eps, beta, k)[0]
        Fm = O.nlc_stokes(lam, b, s, -S, eps, beta, k)[0]
        assert Fp + Fm == pytest.approx(2 * w, rel=1e-13)
        pm = (w - np.linalg.norm(g)) / (2 * w)
        np.testing.assert_allclose((1 - pm) * S - pm * S, g / w, rtol=1e-13)


# ------------------------------------------------------------------------------------------
# Rates: limits and an independent quadrature
# ------------------------------------------------------------------------------------------
def _nlc_rate_scipy(chi, sigma):
    def f(lam):
        up = 2 * lam / (1 - lam) / (3 * chi)
        k13, k23 = sp.kv(1 / 3, up), sp.kv(2 / 3, up)
        ik = si.quad(lambda y: sp.kv(1 / 3, y), up, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
        kap = 1 / (1 - lam) + (1 - lam)
        return -ik + kap * k23 + sigma * lam * k13
    return si.quad(f, 0, 1, epsabs=0, epsrel=1e-10, limit=400, points=[1e-6, 1e-3, 0.1, 0.5, 0.9])[0]


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0])
def test_nlc_rate_against_independent_quadrature(chi):
    for sigma in (1, -1):
        assert O.rate_integral(False, chi, sigma) == pytest.approx(_nlc_rate_scipy(chi, sigma), rel=1e-8)


def test_nbw_rate_against_independent_quadrature():
    chi = 2.0

    def f(lam, sigma):
        ut = 2 * (1 / lam + 1 / (1 - lam)) / (3 * chi)
        k23 = sp.kv(2 / 3, ut)
        ik = si.quad(lambda y: sp.kv(1 / 3, y), ut, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
        rho = (1 - lam) / lam + lam / (1 - lam)
        return ik + rho * k23 - sigma * k23

    for sigma in (1, -1):
        ref = si.quad(lambda l: f(l, sigma), 0, 1, epsabs=0, epsrel=1e-10, limit=400)[0]
        assert O.rate_integral(True, chi, sigma) * math.exp(-8 / (3 * chi)) == pytest.approx(ref, rel=1e-8)


def test_nlc_classical_limit_and_spin_asymmetry():
    """chi -> 0: int (kappa K23 - IntK13) d lambda -> 5 pi chi / 2 (classical photon number,
    using int_0^inf K_{2/3} = pi and int_0^inf x K_{1/3} = pi/3); the spin asymmetry
    (I_up - I_down)/2 = int lambda K13 -> (9 chi^2/4) int x K13 = 3 pi chi^2 / 4."""
    chi = 1e-5
    up, dn = O.rate_integral(False, chi, 1), O.rate_integral(False, chi, -1)
    assert 0.5 * (up + dn) / (2.5 * math.pi * chi) == pytest.approx(1.0, abs=3e-5)
    assert 0.5 * (up - dn) / (0.75 * math.pi * chi * chi) == pytest.approx(1.0, abs=1e-4)
    # the quantum suppression grows with chi
    r = [0.5 * (O.rate_integral(False, c, 1) + O.rate_integral(False, c, -1)) / (2.5 * math.pi * c)
         for c in (1e-3, 0.1, 1.0, 10.0)]
    assert all(a > b for a, b in zip(r, r[1:]))


def test_nbw_small_chi_asymptote_and_polarization_ratio():
    """chi -> 0: J_0 -> 9 pi chi/(16 sqrt2) e^{-8/(3 chi)}, i.e. W = (3 sqrt3/(16 sqrt2)) alpha chi
    e^{-8/(3chi)} / (eta0 eps); the xi3 = -1 state pairs twice as often as xi3 = +1."""
    chi = 0.004
    jp, jm = O.rate_integral(True, chi, 1), O.rate_integral(True, chi, -1)
    assert 0.5 * (jp + jm) / (9 * math.pi * chi / (16 * math.sqrt(2))) == pytest.approx(1.0, abs=2e-3)
    assert jm / jp == pytest.approx(2.0, abs=3e-3)
    assert O.rate_integral(True, 1.0, -1) > O.rate_integral(True, 1.0, 1)


def test_photon_polarization_degree_classical():
    """Number-weighted <xi3> of photons from unpolarized leptons -> 3/5 as chi -> 0
    (int K23 / int (kappa K23 - IntK13) = pi / (5 pi / 3))."""
    chi = 1e-4

    def num(lam):
        up = 2 * lam / (1 - lam) / (3 * chi)
        return O.bessel(up)[1]

    # substitute lambda = (3 chi / 2) t^3 region: integrate in t = u'^{1/3}
    def integ(fun):
        def g(t):
            upp = t ** 3
            lam = 3 * chi * upp / (2 + 3 * chi * upp)
            return fun(lam) * 6 * chi / (2 + 3 * chi * upp) ** 2 * 3 * t * t
        return si.quad(g, 1e-6, 80 ** (1 / 3), epsabs=0, epsrel=1e-10, limit=200)[0]

    ratio = integ(num) / (0.5 * (O.rate_integral(False, chi, 1) + O.rate_integral(False, chi, -1)))
    assert ratio == pytest.approx(0.6, abs=2e-4)


def test_quadrature_rule_converged():
    """Doubling the Gauss-Legendre order and halving the panel width changes nothing at 1e-13."""
    vals = [(False, 0.01, 1), (False, 3.0, -1), (True, 0.3, 1), (True, 30.0, -1)]
    a = [O.rate_integral(*v) for v in vals]
    try:
        O.set_quadrature(20, 1.0 / 32.0)
        b = [O.rate_integral(*v) for v in vals]
    finally:
        O.set_quadrature(10, 1.0 / 16.0)
    np.testing.assert_allclose(a, b, rtol=1e-13)


# ------------------------------------------------------------------------------------------
# Sokolov-Ternov / BKS functions (Sec. 8.1, 8.3)
# ------------------------------------------------------------------------------------------
def _psi_scipy(chi, which):
    def f(u):
        x = 2 * u / (3 * chi)
        upp = u * u / (1 + u) ** 3
        if which == 1:
            return upp * sp.kv(2 / 3, x)
        if which == 3:
            return upp * sp.kv(1 / 3, x)
        ik = si.quad(lambda y: sp.kv(1 / 3, y), x, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
        return upp * (ik - sp.kv(2 / 3, x))
    return si.quad(f, 0, np.inf, epsabs=0, epsrel=1e-10, limit=400)[0]


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0])
def test_psi_against_independent_quadrature(chi):
    for which in (1, 2, 3):
        assert O.psi(chi, which) == pytest.approx(_psi_scipy(chi, which), rel=1e-8)


def test_psi_classical_ratios():
    """chi -> 0: psi3/psi1 -> 8/(5 sqrt3) (the Sokolov-Ternov 92.4 %), psi2/psi1 -> -2/9."""
    chi = 1e-4
    p1, p2, p3 = (O.psi(chi, i) for i in (1, 2, 3))
    assert p3 / p1 == pytest.approx(8 / (5 * math.sqrt(3)), abs=2e-4)
    assert p2 / p1 == pytest.approx(-2 / 9, abs=2e-4)


# ------------------------------------------------------------------------------------------
# Photon polarization vector P (Sec. 3.2)
# ------------------------------------------------------------------------------------------
def test_P_vector_round_trip_and_observation_rotation():
    rng = np.random.default_rng(8)
    eps, beta, k = _rh_basis(8)
    for _ in range(200):
        xi = _unit(rng)[0] * rng.uniform(0, 1)
        P = O.stokes_to_P(xi, eps, beta, k)
        assert np.linalg.norm(P) == pytest.approx(np.linalg.norm(xi), rel=1e-14, abs=1e-15)
        np.testing.assert_allclose(O.P_to_stokes(P, eps, beta, k), xi, atol=1e-14)
        # observation basis rotated by phi (Eq. observation basis): xi1' = xi1 cos2phi - xi3 sin2phi,
        # xi2' = xi2, xi3' = xi1 sin2phi + xi3 cos2phi
        phi = rng.uniform(-math.pi, math.pi)
        o1 = eps * math.cos(phi) + beta * math.sin(phi)
        o2 = -eps * math.sin(phi) + beta * math.cos(phi)
        xo = O.P_to_stokes(P, o1, o2, k)
        c2, s2 = math.cos(2 * phi), math.sin(2 * phi)
        np.testing.assert_allclose(xo, [xi[0] * c2 - xi[2] * s2, xi[1], xi[0] * s2 + xi[2] * c2], atol=1e-13)
