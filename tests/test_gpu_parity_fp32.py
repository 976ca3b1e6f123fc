"""Parity of the FP32 path (FP32 push, lookups and sampling; FP64 optical depth and renormalisation;
the event branch with accurate fields and FP64 where FP32 cancels) with the FP64 oracle on the same
inputs (the oracle starts from the float-rounded state read back from the device).

Bar per step: 1e-5 relative on momenta, spins, Stokes vectors, positions and optical depths, with no
tail: every compared particle is inside it.  Decisions taken in FP32 next to their threshold (the
optical-depth crossing, a collapse sign) may flip: fewer than 1e-5 per particle-step, shown on a run of
4e5 particle-steps.  Over many steps the per-step error compounds at most linearly: an n-step
trajectory is held to n x 1e-5.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_08929_gb300 import binding as B
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import inputs as I

from parity_util import as_oracle_field, as_oracle_step, compare_with_flips, oracle_full_step

pytestmark = pytest.mark.gpu

# the production resolution along r (256 points): the FP32 rounding of the logit coordinate is amplified
# by the slope of the interpolated row, which a coarse grid makes larger
DESC = dict(chi_min=1e-3, chi_max=1e2, n_chi=24, n_r=256, y_lo=-20.0, y_hi=20.0)
ETA0 = I.eta0_for_wavelength(0.8)
FP32 = B.QED_FP32


@pytest.fixture(scope="module")
def gpu_tables():
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    t = Q.Tables(**DESC)
    yield t
    t.close()


@pytest.fixture(scope="module")
def ora_tables():
    return O.tables(*DESC.values())


def _pair(b, charge, cap=None, seed=7, photons=False, use_begin=False):
    """Device buffer (FP32 layout) and an oracle buffer holding the same float-rounded state."""
    n = len(b["id"])
    g = Q.ParticleBuffer(cap or max(n, 1), FP32, charge, photons=photons, use_begin=use_begin)
    g.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    if n:
        g.init_tau(seed)
    r = g.read()
    o = O.Particles.from_arrays(cap or max(n, 1), r["pos"], r["mom"], r["spin"], r["w"], r["id"], tau=r["tau"])
    return g, o


def _run_lepton(gt, ot, b, f, steps, q=-1, flags=None, dt=0.2, t0=8.0, seed=7, cap_ph=400000):
    fl = B.QED_F_FULL if flags is None else flags
    gL, oL = _pair(b, q, seed=seed)
    gG = Q.ParticleBuffer(cap_ph, FP32, B.QED_PHOTON)
    oG = O.Particles(cap_ph)
    ctr, octr = Q.Counters(), O.Counters()
    of = as_oracle_field(f)
    for s in range(steps):
        st = Q.step_desc(dt, t0 + s * dt, s, seed, fl)
        B.qed_push_step(gt.handle, f, st, gL.s, gG.s, ctr.ptr)
        O.lepton_step(ot, of, as_oracle_step(st), q, oL, oG, octr)
    torch.cuda.synchronize()
    return gL, gG, oL, oG, ctr.read(), octr


@pytest.mark.parametrize("n", [1, 33, 4001])
def test_lepton_single_step(gpu_tables, ora_tables, n):
    b = I.random_states(n, seed=200 + n, gamma_range=(50.0, 6000.0), field_region=(-40.0, 10.0))
    f = Q.field(B.QED_FIELD_LP, a0=120.0, n_cycles=5.0, eta0=ETA0)
    for q in (-1, 1):
        gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, 1, q=q, t0=10.0)
        fl1, w1 = compare_with_flips(gL.read(), oL.view(), 1e-5, "leptons")
        fl2, w2 = compare_with_flips(gG.read(), oG.view(), 1e-5, "photons", P_headless=True)
        assert fl1 + fl2 <= 1e-5 * n, (fl1, fl2)
        assert c.status == 0 and int(c.events) == oc.events


def test_flip_rate_per_particle_step(gpu_tables, ora_tables):
    """1e5 leptons of both charges through two steps of a linear laser (4e5 particle-steps, about 8 %
    of them events): every matched particle within the bar, and fewer than 1e-5 decision flips per
    particle-step."""
    n, steps = 100000, 2
    b = I.random_states(n, seed=77, gamma_range=(300.0, 6000.0), field_region=(-40.0, 10.0))
    f = Q.field(B.QED_FIELD_LP, a0=150.0, n_cycles=5.0, eta0=ETA0)
    flips, events = 0, 0
    for q in (-1, 1):
        gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, steps, q=q, t0=10.0, dt=0.15)
        f1, _ = compare_with_flips(gL.read(), oL.view(), 1e-5 * steps, "leptons")
        f2, _ = compare_with_flips(gG.read(), oG.view(), 1e-5 * steps, "photons", P_headless=True)
        flips += f1 + f2
        events += oc.events
    psteps = 2 * n * steps
    assert events > 0.02 * psteps
    assert flips <= 1e-5 * psteps, (flips, psteps, flips / psteps)


def test_emitted_spectrum_error(gpu_tables, ora_tables):
    """Emitted photon energies matched by id: every one within 1e-5 of the oracle's; the spectrum (counts
    on 64 log-spaced bins per decade) identical except for photons within 1e-5 of an edge."""
    b = I.random_states(6000, seed=3, gamma_range=(300.0, 6000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_CP, a0=100.0, n_cycles=4.0, eta0=ETA0)
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, 3)
    g, o = gG.read(), oG.view()
    common, gi, oi = np.intersect1d(g["id"], o["id"], return_indices=True)
    assert len(common) >= 0.999 * oG.n and oG.n > 1000
    eg = np.linalg.norm(g["mom"][gi], axis=1)
    eo = np.linalg.norm(o["mom"][oi], axis=1)
    err = np.abs(eg / eo - 1)
    assert err.max() <= 1e-5, (np.quantile(err, 0.99), err.max())
    edges = 10 ** (np.arange(-8, 4 + 1e-9, 1 / 64))
    hg, _ = np.histogram(eg, edges)
    ho, _ = np.histogram(eo, edges)
    near = np.min(np.abs(np.log(eo[:, None] / edges[None, :])), axis=1) < 1e-5
    assert np.abs(hg - ho).sum() <= 2 * near.sum()


def test_lepton_multi_step(gpu_tables, ora_tables):
    b = I.random_states(2000, seed=5, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_CP, a0=80.0, n_cycles=5.0, eta0=ETA0)
    steps = 40
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, steps, dt=0.1, t0=5.0)
    flips, worst = compare_with_flips(gL.read(), oL.view(), 1e-5 * steps, "leptons")
    pf, _ = compare_with_flips(gG.read(), oG.view(), 1e-5 * steps, "photons", P_headless=True)
    assert flips + pf <= max(2, 1e-5 * 2000 * steps), (flips, pf)


def test_headon_lp_trajectory(gpu_tables, ora_tables):
    wl = I.HEADON_LP_SMALL
    b = wl.beam(n=2000)
    f = Q.laser_field(wl.laser)
    steps = 1300
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, steps, seed=wl.seed, dt=wl.dt, t0=0.0)
    assert oc.events > 5000
    tol = 1e-5 * steps
    flips, worst = compare_with_flips(gL.read(), oL.view(), tol, "leptons", diverged=0.3)
    pf, _ = compare_with_flips(gG.read(), oG.view(), tol, "photons", P_headless=True, diverged=0.3)
    assert flips + pf <= 1e-5 * 2000 * steps, (flips, pf, worst)


@pytest.mark.parametrize("flags", [
    B.QED_F_FULL & ~B.QED_F_TAU,
    B.QED_F_FULL & ~(B.QED_F_SPIN_COLLAPSE | B.QED_F_POL_COLLAPSE),
    B.QED_F_FULL & ~B.QED_F_RESOLVED,
    B.QED_F_FULL | B.QED_F_TBMT_PAPER,
    B.QED_F_FULL & ~B.QED_F_RECOIL,
])
def test_lepton_modes(gpu_tables, ora_tables, flags):
    b = I.random_states(1500, seed=flags % 997, gamma_range=(100.0, 4000.0), field_region=(-30.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=100.0, n_cycles=4.0, eta0=ETA0)
    steps = 4
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, steps, flags=flags, dt=0.15)
    fl1, _ = compare_with_flips(gL.read(), oL.view(), 1e-5 * steps, "leptons")
    fl2, _ = compare_with_flips(gG.read(), oG.view(), 1e-5 * steps, "photons", P_headless=True)
    assert fl1 + fl2 <= max(1, 1e-5 * 1500 * steps)


def _photon_inputs(n, seed, energy=3000.0):
    rng = np.random.default_rng(seed)
    d = np.column_stack([rng.normal(0, 0.05, n), rng.normal(0, 0.05, n), -np.ones(n)])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    e = energy * np.exp(rng.uniform(-1.5, 0.5, n))
    P = rng.normal(size=(n, 3))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    P *= rng.uniform(0, 1, (n, 1))
    pos = np.column_stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-35, 5, n)])
    return {"pos": pos, "mom": d * e[:, None], "spin": P, "w": rng.uniform(0.5, 2, n),
            "id": np.arange(n, dtype=np.uint64) * 104729 + 1}


@pytest.mark.parametrize("flags", [None, B.QED_F_FULL | B.QED_F_BETA_BASIS, B.QED_F_FULL | B.QED_F_REJECT])
def test_photon_pairs_and_compaction(gpu_tables, ora_tables, flags):
    b = _photon_inputs(4000, seed=21)
    f = Q.field(B.QED_FIELD_CP, a0=200.0, n_cycles=4.0, eta0=ETA0)
    of = as_oracle_field(f)
    gG, oG = _pair(b, B.QED_PHOTON, seed=4, photons=True)
    gE, gP = Q.ParticleBuffer(8000, FP32, B.QED_ELECTRON), Q.ParticleBuffer(8000, FP32, B.QED_POSITRON)
    oE, oP = O.Particles(8000), O.Particles(8000)
    ws = Q.CompactWorkspace(gG.capacity)
    ctr, octr = Q.Counters(), O.Counters()
    steps = 20
    for s in range(steps):
        st = Q.step_desc(0.2, 6.0 + 0.2 * s, s, 4, flags)
        B.qed_pair_step(gpu_tables.handle, f, st, gG.s, gE.s, gP.s, ctr.ptr)
        B.qed_compact(gG.s, ws.ptr, ws.bytes)
        O.photon_step(ora_tables, of, as_oracle_step(st), oG, oE, oP, octr)
    torch.cuda.synchronize()
    assert octr.events > 200 and ctr.read().status == 0
    # photons are held to the n-step bar, and so are their daughters: a pair made at step k inherits its
    # photon's k-step state (pairs made from the same state in one step: test_gpu_overflow, at 1e-5).
    # P is compared headless: a photon without pair rate keeps its P as loaded, the oracle rewrites it in
    # its own representative (P and -P_perp are the same Stokes vector)
    f1, _ = compare_with_flips(gG.read(), oG.view(), 1e-5 * steps, "photons", P_headless=True)
    f2, _ = compare_with_flips(gE.read(), oE.view(), 1e-5 * steps, "electrons")
    f3, _ = compare_with_flips(gP.read(), oP.view(), 1e-5 * steps, "positrons")
    assert f1 + f2 + f3 <= max(1, 1e-5 * 4000 * steps), (f1, f2, f3)


def test_soft_photons_move_along_k(gpu_tables, ora_tables):
    """Photons down to 1e-30 mc^2 (the NLC spectrum's lambda^(1/3) tail stores a few per 1e8 emissions
    below 1e-15): |k|^2 leaves the float range, yet each moves by dt k-hat like the oracle's, to 1e-6 of
    the position (and keeps its k, P and optical depth); the FULL-flag step, in and out of the pulse."""
    n = 400
    rng = np.random.default_rng(5)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    e = 10.0 ** rng.uniform(-30.0, 2.0, n)
    pos = np.column_stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-40, 10, n)])
    b = {"pos": pos, "mom": d * e[:, None], "spin": np.zeros((n, 3)), "w": np.ones(n),
         "id": np.arange(n, dtype=np.uint64) * 7 + 3}
    f = Q.field(B.QED_FIELD_LP, a0=150.0, n_cycles=4.0, eta0=ETA0)
    gG, oG = _pair(b, B.QED_PHOTON, seed=9, photons=True)
    gE, gP = Q.ParticleBuffer(64, FP32, B.QED_ELECTRON), Q.ParticleBuffer(64, FP32, B.QED_POSITRON)
    oE, oP = O.Particles(64), O.Particles(64)
    ctr, octr = Q.Counters(), O.Counters()
    st = Q.step_desc(0.2, 6.0, 0, 9)
    B.qed_pair_step(gpu_tables.handle, f, st, gG.s, gE.s, gP.s, ctr.ptr)
    O.photon_step(ora_tables, as_oracle_field(f), as_oracle_step(st), oG, oE, oP, octr)
    torch.cuda.synchronize()
    g, o = gG.read(), oG.view()
    assert ctr.read().events == 0 and octr.events == 0 and len(g["id"]) == n
    go, oo = np.argsort(g["id"]), np.argsort(o["id"])
    dx = np.linalg.norm(g["pos"][go] - o["pos"][oo], axis=1) / np.maximum(np.linalg.norm(o["pos"][oo], axis=1), 1.0)
    assert dx.max() < 1e-6, (dx.max(), e[go][np.argmax(dx)])
    np.testing.assert_array_equal(g["mom"][go], o["mom"][oo].astype(np.float32).astype(np.float64))
    # every photon moved by dt (the soft ones too)
    moved = np.linalg.norm(g["pos"][go] - b["pos"][go].astype(np.float32), axis=1)
    assert np.all(np.abs(moved - 0.2) < 1e-5)


def test_constant_field_general_forms(gpu_tables, ora_tables):
    """A constant field with every component nonzero: the FP32 path takes the general forms of chi, the
    basis vector, the Boris push and the T-BMT vector here (the plane-wave forms do not apply)."""
    f = Q.field(B.QED_FIELD_CONST, E0=(20.0, -15.0, 10.0), B0=(12.0, 25.0, -18.0), eta0=ETA0)
    b = I.random_states(3000, seed=41, gamma_range=(300.0, 6000.0), field_region=(-5.0, 5.0))
    steps = 3
    for q in (-1, 1):
        gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, steps, q=q, t0=0.0)
        assert oc.events > 20 and c.status == 0
        fl1, _ = compare_with_flips(gL.read(), oL.view(), 1e-5 * steps, "leptons")
        fl2, _ = compare_with_flips(gG.read(), oG.view(), 1e-5 * steps, "photons", P_headless=True)
        assert fl1 + fl2 <= 1, (fl1, fl2)
    pb = _photon_inputs(3000, seed=43, energy=20000.0)
    gG, oG = _pair(pb, B.QED_PHOTON, seed=5, photons=True)
    gE, gP = Q.ParticleBuffer(6000, FP32, B.QED_ELECTRON), Q.ParticleBuffer(6000, FP32, B.QED_POSITRON)
    oE, oP = O.Particles(6000), O.Particles(6000)
    ctr, octr = Q.Counters(), O.Counters()
    ws = Q.CompactWorkspace(gG.capacity)
    of = as_oracle_field(f)
    for s_ in range(steps):
        st = Q.step_desc(0.2, 0.2 * s_, s_, 5)
        B.qed_pair_step(gpu_tables.handle, f, st, gG.s, gE.s, gP.s, ctr.ptr)
        B.qed_compact(gG.s, ws.ptr, ws.bytes)  # converted photons leave, as in the oracle's step
        O.photon_step(ora_tables, of, as_oracle_step(st), oG, oE, oP, octr)
    torch.cuda.synchronize()
    assert ctr.read().status == 0
    # P is headless: its transverse part is fixed only up to sign (the representative with P.eps >= 0),
    # and a photon whose P is nearly perpendicular to eps may land on either side in FP32 and FP64
    f1, _ = compare_with_flips(gG.read(), oG.view(), 1e-5 * steps, "photons", P_headless=True)
    f2, _ = compare_with_flips(gE.read(), oE.view(), 1e-5 * steps, "electrons")
    f3, _ = compare_with_flips(gP.read(), oP.view(), 1e-5 * steps, "positrons")
    assert f1 + f2 + f3 <= 1, (f1, f2, f3)


def test_coupled_species(gpu_tables, ora_tables):
    f = Q.field(B.QED_FIELD_CP_COUNTER, a0=300.0, n_cycles=3.0, phase=3 * math.pi - 4.0,
                eta0=I.eta0_for_wavelength(1.0))
    of = as_oracle_field(f)
    b = I.lepton_beam(400, 1000.0, direction=(1, 0, 0), z_range=(-0.5, 0.5), spin="random", seed=31)
    cap = 60000
    gE, oE = _pair(b, B.QED_ELECTRON, cap=cap, seed=31, use_begin=True)
    gPo = Q.ParticleBuffer(cap, FP32, B.QED_POSITRON, use_begin=True)
    gG = Q.ParticleBuffer(cap, FP32, B.QED_PHOTON, photons=True, use_begin=True)
    oPo, oG = O.Particles(cap), O.Particles(cap)
    ws = Q.CompactWorkspace(cap)
    ctr = Q.Counters()
    steps = 50
    for s in range(steps):
        st = Q.step_desc(0.1, 0.1 * s, s, 31, B.QED_F_FULL, photon_store_min=2.0)
        B.qed_snapshot_counts([gE.s, gPo.s, gG.s])
        B.qed_pair_step(gpu_tables.handle, f, st, gG.s, gE.s, gPo.s, ctr.ptr)
        B.qed_push_step(gpu_tables.handle, f, st, gE.s, gG.s, ctr.ptr)
        B.qed_push_step(gpu_tables.handle, f, st, gPo.s, gG.s, ctr.ptr)
        B.qed_compact(gG.s, ws.ptr, ws.bytes)
        oracle_full_step(ora_tables, of, as_oracle_step(st), [(oE, -1), (oPo, 1)], oG, oE, oPo)
    torch.cuda.synchronize()
    assert oG.n > 100
    tol = 1e-5 * steps
    f1, _ = compare_with_flips(gE.read(), oE.view(), tol, "electrons")
    f2, _ = compare_with_flips(gPo.read(), oPo.view(), tol, "positrons")
    f3, _ = compare_with_flips(gG.read(), oG.view(), tol, "photons", P_headless=True)
    psteps = steps * (oE.n + oG.n)
    assert f1 + f2 + f3 <= max(4, 1e-5 * psteps), (f1, f2, f3)
