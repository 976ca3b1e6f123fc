"""Pins of the oracle's step functions: exact discrete dynamics (Boris, T-BMT), conservation at
events, invariants, the ICDF against the exact CDF, and the paper's verification experiments
reduced to 0-D with analytic fields: Sokolov-Ternov (Sec. 6 and 8.1) and the construction
independence of unpolarized photon beams under the non-pair update (Sec. 6).  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2511_08929_gb300 import inputs as I

ALPHA = 7.2973525693e-3
AE = ALPHA / (2 * math.pi)
ETA0 = I.eta0_for_wavelength(0.8)
GAMMA_1GEV = 1e9 / I.ME_EV


def _particles(b, cap=None, seed=None):
    n = len(b["id"])
    p = O.Particles.from_arrays(cap or n, b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    if seed is not None:
        p.init_tau(seed)
    return p


# ------------------------------------------------------------------------------------------
# exact discrete dynamics
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("q", [-1, 1])
def test_boris_gyration_angle_exact(q, small_tables):
    """E = 0, uniform B: the Boris step rotates p about B by 2 atan(q B dt / (2 gamma)) exactly."""
    g, Bz, dt, n = 300.0, 40.0, 0.07, 250
    pm = math.sqrt(g * g - 1)
    b = {"pos": np.zeros((1, 3)), "mom": np.array([[pm, 0, 0]]), "spin": np.array([[0, 0, 1.0]]),
         "w": np.ones(1), "id": np.array([1], dtype=np.uint64)}
    L = _particles(b)
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    for s in range(n):
        O.lepton_step(small_tables, f, O.step_desc(dt, s * dt, s, 1, O.F_PUSH | O.F_MOVE), q, L, None)
    th = -q * n * 2 * math.atan(Bz * dt / (2 * g))  # dp/dt = (-q B/gamma) z x p
    v = L.view()["mom"][0]
    np.testing.assert_allclose(v, [pm * math.cos(th), pm * math.sin(th), 0.0], rtol=0, atol=1e-11 * pm)


def test_tbmt_precession_relative_to_momentum(small_tables):
    """Uniform B, p and s in the plane: s rotates by (a + 1/gamma_bar) B dt per step (gamma_bar from the
    time-centred momentum), so s advances against p at a gamma omega_c to O(dt^2) (T-BMT, Sec. 8.3)."""
    g, Bz, dt, n = 50.0, 10.0, 0.05, 400
    pm = math.sqrt(g * g - 1)
    b = {"pos": np.zeros((1, 3)), "mom": np.array([[pm, 0, 0]]), "spin": np.array([[1.0, 0, 0]]),
         "w": np.ones(1), "id": np.array([3], dtype=np.uint64)}
    L = _particles(b)
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    for s in range(n):
        O.lepton_step(small_tables, f, O.step_desc(dt, s * dt, s, 1, O.F_PUSH | O.F_TBMT | O.F_MOVE), -1, L, None)
    th_p = 2 * math.atan(Bz * dt / (2 * g))
    gbar = math.sqrt(1 + (pm * math.cos(th_p / 2)) ** 2)
    th_s = (AE + 1 / gbar) * Bz * dt
    v = L.view()
    ang_p = math.atan2(v["mom"][0][1], v["mom"][0][0])
    ang_s = math.atan2(v["spin"][0][1], v["spin"][0][0])
    rel = (ang_s - ang_p + math.pi) % (2 * math.pi) - math.pi
    exact = ((n * (th_s - th_p)) + math.pi) % (2 * math.pi) - math.pi
    assert rel == pytest.approx(exact, abs=1e-10)
    # continuum limit: the relative angle grows at a gamma omega_c = a B
    assert n * (th_s - th_p) == pytest.approx(AE * Bz * n * dt, rel=2e-3)


# ------------------------------------------------------------------------------------------
# conservation and invariants at events
# ------------------------------------------------------------------------------------------
def test_momentum_conservation_nlc_and_invariants(small_tables):
    """No classical force: every emission satisfies p_i = p_f + hbar k exactly (Sec. 5.1), |s| <= 1,
    |P| <= 1 for every particle after many steps."""
    b = I.random_states(400, seed=11)
    L = _particles(b, seed=5)
    G = O.Particles(100000)
    f = O.field(O.FIELD_CONST, E0=(0, 0, 0), B0=(30.0, 10.0, 0.0), eta0=ETA0)
    p0 = L.view()["mom"].sum(0)
    fl = O.F_FULL & ~O.F_PUSH & ~O.F_TBMT
    ctr = O.Counters()
    for s in range(300):
        O.lepton_step(small_tables, f, O.step_desc(0.05, 0.05 * s, s, 5, fl), -1, L, G, ctr)
    assert ctr.events > 1000 and ctr.dropped_capacity == 0
    v, gv = L.view(), G.view()
    tot = v["mom"].sum(0) + gv["mom"].sum(0)
    np.testing.assert_allclose(tot, p0, rtol=0, atol=1e-10 * np.abs(p0).max())
    assert np.linalg.norm(v["spin"], axis=1).max() <= 1.0 + 1e-14
    assert np.linalg.norm(gv["spin"], axis=1).max() <= 1.0 + 1e-14
    assert len(np.unique(gv["id"])) == G.n  # daughter ids are distinct


def test_nbw_momentum_conservation_and_spins(small_tables):
    """p_e + p_p = hbar k for every pair (Sec. 5.2); daughters' spins are unit (four-state collapse)."""
    eps_ = 4000.0
    P_list = [(0, 1, 0), (0, 0, 1), (1, 0, 0), (0, 0.7, 0.7)]
    b = I.photon_beam(2000, eps_, direction=(1, 0, 0), P_list=P_list, seed=3)
    G = _particles(b, seed=7)
    el, po = O.Particles(5000), O.Particles(5000)
    Bz = 3.0 / (ETA0 * eps_)  # chi_gamma = 3
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    k_by_id = {int(i): m for i, m in zip(b["id"], b["mom"])}
    ctr = O.Counters()
    for s in range(60):
        O.photon_step(small_tables, f, O.step_desc(0.2, 0.2 * s, s, 7), G, el, po, ctr)
    assert ctr.events > 200 and el.n == po.n == ctr.events
    ev, pv = el.view(), po.view()
    np.testing.assert_allclose(ev["mom"] + pv["mom"], np.tile([eps_, 0, 0], (el.n, 1)), rtol=1e-14, atol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(ev["spin"], axis=1), 1.0, rtol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(pv["spin"], axis=1), 1.0, rtol=1e-13)
    assert G.n + el.n == 2000
    assert len(k_by_id) == 2000


# ------------------------------------------------------------------------------------------
# sampling: the tabulated ICDF against the exact CDF (Sec. 4.2, 5.1, 5.2)
# ------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def node_tables():
    return O.tables(0.05, 50.0, 4, 256)


@pytest.mark.parametrize("nbw", [False, True])
def test_icdf_on_grid_rows_matches_exact_cdf(nbw, node_tables):
    tb = node_tables
    chis = [0.05, 0.05 * 10 ** 1, 50.0]
    rs = np.concatenate([np.logspace(-8, -1, 8), np.linspace(0.1, 0.9, 9), 1 - np.logspace(-1, -7, 7)])
    for chi in chis:
        for s, sigma in ((0, 1), (1, -1)):
            for r in rs:
                v = math.exp(tb.icdf(nbw, s, chi, r))
                t = math.sqrt(v) if nbw else v ** (1 / 3)
                c = O.cdf_t(nbw, chi, sigma, t)
                assert abs(c - r) <= 1e-6 + 2e-6 * min(r, 1 - r), (chi, sigma, r, c)


def test_icdf_between_rows_and_rate_interpolation(small_tables):
    """Between chi nodes the rows are blended linearly in ln chi: errors stay at the 1e-3 level on
    the coarse 24-row test grid, and the rate lookups are exact on nodes."""
    tb = small_tables
    d = tb.desc
    dl = (math.log(d.chi_max) - math.log(d.chi_min)) / (d.n_chi - 1)
    for i in (3, 11, 19):
        chi = math.exp(math.log(d.chi_min) + i * dl)
        assert tb.nlc_rate_lookup(0, chi) == pytest.approx(O.rate_integral(False, chi, 1), rel=1e-13)
        assert tb.nbw_rate_lookup(1, chi) == pytest.approx(
            O.rate_integral(True, chi, -1) * math.exp(-8 / (3 * chi)), rel=1e-12)
        chim = math.exp(math.log(d.chi_min) + (i + 0.5) * dl)
        assert tb.nlc_rate_lookup(0, chim) == pytest.approx(O.rate_integral(False, chim, 1), rel=3e-3)
        for r in (0.01, 0.3, 0.8, 0.99):
            up = math.exp(tb.icdf(False, 1, chim, r))
            assert O.cdf_t(False, chim, -1, up ** (1 / 3)) == pytest.approx(r, abs=5e-3)
    # below chi_min the NLC rate is classical (proportional to chi); above chi_max it is clamped
    c = d.chi_min / 10
    assert tb.nlc_rate_lookup(0, c) == pytest.approx(tb.nlc_rate_lookup(0, d.chi_min) / 10, rel=1e-14)
    assert tb.nlc_rate_lookup(0, 10 * d.chi_max) == pytest.approx(tb.nlc_rate_lookup(0, d.chi_max), rel=1e-14)
    assert tb.nbw_rate_lookup(0, d.chi_min / 2) == 0.0


def test_sampled_spectrum_is_the_spin_mixture(small_tables):
    """Branch choice with weights W_up(1+s)/2, W_down(1-s)/2 then the branch ICDF reproduces the CDF
    of w(lambda; s_beta) exactly in distribution (w is linear in s_beta): check with stratified r."""
    tb = small_tables
    d = tb.desc
    dl = (math.log(d.chi_max) - math.log(d.chi_min)) / (d.n_chi - 1)
    chi = math.exp(math.log(d.chi_min) + 14 * dl)
    sb = 0.6
    Iu, Id = O.rate_integral(False, chi, 1), O.rate_integral(False, chi, -1)
    wu, wd = Iu * (1 + sb) / 2, Id * (1 - sb) / 2
    M = 4000
    lam = []
    for m in range(M):
        r = (m + 0.5) / M
        # split the unit interval: [0, wd/(wu+wd)) -> down branch, rest -> up, each re-scaled to (0, 1)
        pdn = wd / (wu + wd)
        if r < pdn:
            up = math.exp(tb.icdf(False, 1, chi, r / pdn))
        else:
            up = math.exp(tb.icdf(False, 0, chi, (r - pdn) / (1 - pdn)))
        lam.append(O.nlc_lambda(chi, up))
    lam = np.sort(lam)
    # exact mixture CDF at a few quantiles
    for q in (0.1, 0.5, 0.9):
        l = lam[int(q * M)]
        up = 2 * l / (1 - l) / (3 * chi)
        t = up ** (1 / 3)
        c = (wu * O.cdf_t(False, chi, 1, t) + wd * O.cdf_t(False, chi, -1, t)) / (wu + wd)
        assert c == pytest.approx(q, abs=2e-3)


# ------------------------------------------------------------------------------------------
# Sokolov-Ternov (Sec. 6 first example; Sec. 8.1)
# ------------------------------------------------------------------------------------------
def _st_run(q, n, steps, dt, flags, tables, seed=21):
    p = math.sqrt(GAMMA_1GEV ** 2 - 1)
    Bz = 1.0 / (ETA0 * p)  # chi = eta0 |p x B| = 1
    b = I.lepton_beam(n, GAMMA_1GEV, direction=(1, 0, 0), spin="random", seed=seed)
    L = _particles(b, seed=seed)
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    out = []
    for s in range(steps):
        O.lepton_step(tables, f, O.step_desc(dt, s * dt, s, seed, flags), q, L, None)
        if (s + 1) % (steps // 4) == 0:
            out.append(((s + 1) * dt, L.view()["spin"][:, 2].mean()))
    return out


@pytest.fixture(scope="module")
def st_tables():
    return O.tables(0.5, 2.0, 3, 128)


def test_sokolov_ternov_equilibrium_and_rate(st_tables):
    """1 GeV electrons gyrating in a 2.26 MT-equivalent field (chi = 1), radiation reaction off:
    <S_z>(t) = -(psi3/psi1)(1 - exp(-Gamma psi1 t)), Gamma = alpha/(sqrt3 pi eta0 gamma).  The
    closed form follows from summing the emission expectation g and the non-emission update."""
    fl = O.F_FULL & ~O.F_RECOIL
    # W dt = 0.032: the scheme's O(W dt) bias (0.046 at dt = 0.1, 0.024 at 0.05) is below the noise here
    n, steps, dt = 20000, 1600, 0.025
    res = _st_run(-1, n, steps, dt, fl, st_tables)
    p1, p3 = O.psi(1.0, 1), O.psi(1.0, 3)
    gam = ALPHA / (math.sqrt(3) * math.pi * ETA0 * GAMMA_1GEV)
    for t, sz in res:
        exact = -(p3 / p1) * (1 - math.exp(-gam * p1 * t))
        assert sz == pytest.approx(exact, abs=0.02), (t, sz, exact)
    # without the non-emission update the equilibrium is wrong (Fig. 5, blue curve)
    res2 = _st_run(-1, n, 800, 0.05, fl & ~O.F_NONTRANSITION, st_tables)
    t, sz = res2[-1]
    assert abs(sz + (p3 / p1) * (1 - math.exp(-gam * p1 * t))) > 0.1


def test_sokolov_ternov_positrons_polarize_along_B(st_tables):
    fl = O.F_FULL & ~O.F_RECOIL
    res = _st_run(+1, 6000, 1600, 0.025, fl, st_tables, seed=22)
    p1, p3 = O.psi(1.0, 1), O.psi(1.0, 3)
    gam = ALPHA / (math.sqrt(3) * math.pi * ETA0 * GAMMA_1GEV)
    t, sz = res[-1]
    assert sz == pytest.approx((p3 / p1) * (1 - math.exp(-gam * p1 * t)), abs=0.04)


# ------------------------------------------------------------------------------------------
# unpolarized photon beams built three ways (Sec. 6, second example)
# ------------------------------------------------------------------------------------------
def _nopair_run(construction, flags, tables, n=20000, steps=300, dt=0.1):
    eps_ = GAMMA_1GEV
    Bz = 1.0 / (ETA0 * eps_)  # chi_gamma = 1
    # photon along +x in B_z: eps_hat = -y, beta_hat = k x eps = -z (electron convention)
    ex, bz = np.array([0, -1.0, 0]), np.array([0, 0, -1.0])
    pairs = {"linear": (ex, bz), "circular": (np.array([1.0, 0, 0]), np.array([-1.0, 0, 0])),
             "diagonal": ((ex + bz) / math.sqrt(2), (ex - bz) / math.sqrt(2))}[construction]
    b = I.photon_beam(n, eps_, direction=(1, 0, 0), P_list=list(pairs), seed=5)
    G = _particles(b, seed=31)
    el, po = O.Particles(n), O.Particles(n)
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    for s in range(steps):
        O.photon_step(tables, f, O.step_desc(dt, s * dt, s, 31, flags), G, el, po)
    v = G.view()
    xi = np.array([O.P_to_stokes(P, ex, bz, np.array([1.0, 0, 0])) for P in v["spin"]])
    return xi[:, 2].mean(), G.n


@pytest.mark.slow
def test_unpolarized_photon_beams_evolve_identically(st_tables):
    fl = O.F_FULL
    m = {c: _nopair_run(c, fl, st_tables) for c in ("linear", "circular", "diagonal")}
    vals = [v[0] for v in m.values()]
    assert min(v[1] for v in m.values()) < 19000  # pairs were made
    assert max(vals) - min(vals) < 0.025, m
    assert min(vals) > 0.02  # xi3 = -1 is depleted, the surviving beam drifts to xi3 > 0
    # without the non-pair update the circular construction cannot move
    m2 = {c: _nopair_run(c, fl & ~O.F_NONTRANSITION, st_tables) for c in ("linear", "circular")}
    assert abs(m2["circular"][0]) < 0.01 and m2["linear"][0] > 0.02


# ------------------------------------------------------------------------------------------
# buffer overflow: an event whose daughters find no slot is not applied (Sec. 4.3, reading R2)
# ------------------------------------------------------------------------------------------
def test_overflow_emission_not_applied(small_tables):
    """No classical force, every lepton close to its optical-depth crossing.  One step with room for
    every photon (run A) against one with room for half of them (run B): the first half of the
    emitters (parent order) end as in A; each refused emitter keeps its initial momentum and spin, which
    is A's recoiled momentum plus A's photon (p_i = p_f + hbar k, Sec. 5.1), and a spent optical depth,
    so it emits in the next step.  A rule that applied the recoil or discarded the photon fails here."""
    b = I.random_states(400, seed=21)
    tau0 = np.full(400, 1e-4)
    f = O.field(O.FIELD_CONST, E0=(0, 0, 0), B0=(30.0, 10.0, 0.0), eta0=ETA0)
    fl = O.F_FULL & ~O.F_PUSH & ~O.F_TBMT
    st = O.step_desc(0.05, 0.0, 0, 9, fl)

    def run(cap):
        L = O.Particles.from_arrays(400, b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=tau0)
        G = O.Particles(cap)
        return L, G, O.lepton_step(small_tables, f, st, -1, L, G)

    LA, GA, cA = run(100000)
    va, ga = LA.view(), GA.view()
    emit = np.flatnonzero(np.any(va["mom"] != b["mom"], axis=1))
    nA = len(emit)
    assert cA.events == nA == GA.n and nA > 50 and cA.dropped_capacity == 0
    c = nA // 2
    LB, GB, cB = run(c)
    vb, gb = LB.view(), GB.view()
    assert cB.events == c and cB.dropped_capacity == nA - c and GB.n == c
    # the photons that fit and their emitters are those of run A
    for k in ("pos", "mom", "spin", "tau", "id"):
        np.testing.assert_array_equal(gb[k], ga[k][:c])
    applied, refused = emit[:c], emit[c:]
    quiet = np.setdiff1d(np.arange(400), emit)
    for k in ("pos", "mom", "spin", "tau"):
        np.testing.assert_array_equal(vb[k][applied], va[k][applied])
        np.testing.assert_array_equal(vb[k][quiet], va[k][quiet])
    # refused emitters: the pre-event state, equal to A's recoil plus A's photon
    np.testing.assert_array_equal(vb["mom"][refused], b["mom"][refused])
    np.testing.assert_array_equal(vb["spin"][refused], b["spin"][refused])
    pk = va["mom"][refused] + ga["mom"][c:]
    np.testing.assert_allclose(pk, vb["mom"][refused], rtol=0,
                               atol=1e-12 * np.abs(vb["mom"][refused]).max())
    assert np.all(vb["tau"][refused] <= 0.0) and np.all(va["tau"][applied] > 0.0)
    # with room in the next step every refused emitter emits
    G2 = O.Particles(100000)
    O.lepton_step(small_tables, f, O.step_desc(0.05, 0.05, 1, 9, fl), -1, LB, G2)
    v2 = LB.view()
    assert np.all(np.any(v2["mom"][refused] != b["mom"][refused], axis=1))


def test_overflow_pair_not_applied(small_tables):
    """Photons at chi_gamma = 3, each close to its optical-depth crossing, with room for half of the
    pairs: the first half of the converting photons (parent order) are removed and their pairs carry
    k (p_e + p_p = hbar k, Sec. 5.2); every other converting photon survives with its k and P unchanged
    and a spent optical depth, and converts in the next step once there is room.  No pair is split."""
    eps_ = 4000.0
    b = I.photon_beam(600, eps_, direction=(1, 0, 0), P_list=[(0, 1, 0), (0, 0, 1)], seed=5)
    Bz = 3.0 / (ETA0 * eps_)
    f = O.field(O.FIELD_CONST, B0=(0, 0, Bz), eta0=ETA0)
    st = O.step_desc(0.2, 0.0, 0, 7)
    tau0 = np.full(600, 1e-6)

    def run(cap_e, cap_p):
        G = O.Particles.from_arrays(600, b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=tau0)
        el, po = O.Particles(cap_e), O.Particles(cap_p)
        return G, el, po, O.photon_step(small_tables, f, st, G, el, po)

    GA, elA, poA, cA = run(5000, 5000)
    nA = cA.events
    assert nA > 50 and elA.n == poA.n == nA and GA.n == 600 - nA
    c = nA // 2
    GB, elB, poB, cB = run(5000, c)  # the positron buffer is the short one
    assert cB.events == c and cB.dropped_capacity == nA - c and elB.n == poB.n == c
    gav, gbv = GA.view(), GB.view()
    ea, eb, pa, pb = elA.view(), elB.view(), poA.view(), poB.view()
    for k in ("pos", "mom", "spin", "tau", "id"):
        np.testing.assert_array_equal(eb[k], ea[k][:c])
        np.testing.assert_array_equal(pb[k], pa[k][:c])
    np.testing.assert_allclose(eb["mom"] + pb["mom"], np.tile([eps_, 0, 0], (c, 1)), rtol=1e-14, atol=1e-9)
    # the photons of run A's second half of pairs survive in B, unchanged but for x and tau
    gone_a = set(int(i) for i in b["id"]) - set(int(i) for i in gav["id"])
    left_b = {int(i): j for j, i in enumerate(gbv["id"])}
    refused = [i for i in gone_a if i in left_b]
    assert len(refused) == nA - c and GB.n == 600 - c
    row = {int(i): j for j, i in enumerate(b["id"])}
    for i in refused:
        jb, j0 = left_b[i], row[i]
        np.testing.assert_array_equal(gbv["mom"][jb], b["mom"][j0])
        np.testing.assert_array_equal(gbv["spin"][jb], b["spin"][j0])
        assert gbv["tau"][jb] <= 0.0
    el2, po2 = O.Particles(5000), O.Particles(5000)
    c2 = O.photon_step(small_tables, f, O.step_desc(0.2, 0.2, 1, 7), GB, el2, po2)
    assert c2.events >= len(refused)
    left2 = set(int(i) for i in GB.view()["id"])
    assert not (set(refused) & left2)
