"""Parity of the plain FP64 CUDA path with the FP64 oracle, element by element on the same seeded
inputs, matched by particle id.  Tolerance 1e-12 relative per step (the FP64 bar); longer trajectories
get the per-step bar times the step count (rounding differences of the two libms add up linearly)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_08929_gb300 import binding as B
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import inputs as I

from parity_util import (as_oracle_field, as_oracle_step, compare_sets, gpu_particles, oracle_full_step,
                         oracle_particles)

pytestmark = pytest.mark.gpu

DESC = dict(chi_min=1e-3, chi_max=1e2, n_chi=24, n_r=64, y_lo=-20.0, y_hi=20.0)
ETA0 = I.eta0_for_wavelength(0.8)
FP64 = B.QED_FP64


@pytest.fixture(scope="module")
def gpu_tables():
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    assert torch.cuda.is_available()
    t = Q.Tables(**DESC)
    yield t
    t.close()


@pytest.fixture(scope="module")
def ora_tables():
    return O.tables(DESC["chi_min"], DESC["chi_max"], DESC["n_chi"], DESC["n_r"], DESC["y_lo"], DESC["y_hi"])


# ------------------------------------------------------------------------------------------------
# tables, special functions, lookups
# ------------------------------------------------------------------------------------------------
def test_tables_match_oracle(gpu_tables, ora_tables):
    g = gpu_tables.export()
    np.testing.assert_allclose(g["nlc_rate"], ora_tables.nlc_rate, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g["nbw_rate"], ora_tables.nbw_rate, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g["nlc_icdf"], ora_tables.nlc_icdf, rtol=0, atol=2e-11)
    np.testing.assert_allclose(g["nbw_icdf"], ora_tables.nbw_icdf, rtol=0, atol=2e-11)


def test_bessel_device_matches_oracle(gpu_tables):
    rng = np.random.default_rng(1)
    x = np.concatenate([np.logspace(-12, 4.3, 300), np.exp(rng.uniform(math.log(1e-9), math.log(3e4), 300))])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    ref = np.array([O.bessel(v, scaled=True) for v in x])
    for prec, tol in ((B.QED_FP64, 2e-14), (B.QED_FP32, 4e-6)):
        out = torch.zeros(3 * len(x), dtype=torch.float64, device="cuda")
        B.qed_bessel_eval(gpu_tables.handle, prec, xd.data_ptr(), out.data_ptr(), len(x))
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1, 3)
        if prec == B.QED_FP32:  # the FP32 table spans x < 3e4; float exp underflows nothing at these arguments
            sel = x < 2.9e4
            got, r = got[sel], ref[sel]
        else:
            r = ref
        err = np.abs(got / r - 1).max()
        assert err <= tol, (prec, err)


def test_lookups_match_oracle(gpu_tables, ora_tables):
    rng = np.random.default_rng(2)
    n = 2000
    chi = np.exp(rng.uniform(math.log(2e-4), math.log(3e2), n))  # includes below chi_min and above chi_max
    r = np.concatenate([rng.uniform(0, 1, n - 6), [1e-12, 1e-9, 0.5, 1 - 1e-9, 1 - 1e-12, 0.999]])
    out = torch.zeros(B.QED_LOOKUP_COLS * n, dtype=torch.float64, device="cuda")
    cd = torch.tensor(chi, device="cuda")
    rd = torch.tensor(r, device="cuda")
    B.qed_tables_lookup(gpu_tables.handle, FP64, cd.data_ptr(), rd.data_ptr(), out.data_ptr(), n)
    torch.cuda.synchronize()
    g = out.cpu().numpy().reshape(n, -1)
    for i in range(n):
        ref = [ora_tables.nlc_rate_lookup(0, chi[i]), ora_tables.nlc_rate_lookup(1, chi[i]),
               ora_tables.nbw_rate_lookup(0, chi[i]), ora_tables.nbw_rate_lookup(1, chi[i])]
        np.testing.assert_allclose(g[i, :2], ref[:2], rtol=1e-13, atol=1e-300)
        # NBW rates are exp(L - 8/(3 chi)): compare logs; a 1e-16 relative error in a large exponent is
        # an absolute error |exponent| * 1e-16 in the log
        if ref[2] > 0:
            lg, lr = np.log(g[i, 2:4]), np.log(ref[2:4])
            assert np.all(np.abs(lg - lr) <= 1e-13 + 4e-16 * np.abs(lr)), (chi[i], lg, lr)
        else:
            assert g[i, 2] == 0 and g[i, 3] == 0
        ic = [ora_tables.icdf(False, 0, chi[i], r[i]), ora_tables.icdf(False, 1, chi[i], r[i]),
              ora_tables.icdf(True, 0, chi[i], r[i]), ora_tables.icdf(True, 1, chi[i], r[i])]
        np.testing.assert_allclose(g[i, 4:8], ic, rtol=0, atol=1e-12 * max(1.0, np.abs(ic).max()))


# ------------------------------------------------------------------------------------------------
# lepton step
# ------------------------------------------------------------------------------------------------
def _run_lepton(gpu_tables, ora_tables, b, f, steps, q=-1, flags=None, dt=2 * math.pi / 100, t0=0.0, seed=7,
                cap_ph=200000, store_min=0.0):
    fl = B.QED_F_FULL if flags is None else flags
    gL = gpu_particles(b, FP64, q, seed=seed)
    gG = Q.ParticleBuffer(cap_ph, FP64, B.QED_PHOTON)
    oL = oracle_particles(b, seed=seed)
    oG = O.Particles(cap_ph)
    ctr = Q.Counters()
    octr = O.Counters()
    of = as_oracle_field(f)
    for s in range(steps):
        st = Q.step_desc(dt, t0 + s * dt, s, seed, fl, photon_store_min=store_min)
        B.qed_push_step(gpu_tables.handle, f, st, gL.s, gG.s, ctr.ptr)
        O.lepton_step(ora_tables, of, as_oracle_step(st), q, oL, oG, octr)
    torch.cuda.synchronize()
    return gL, gG, oL, oG, ctr.read(), octr


@pytest.mark.parametrize("n", [1, 33, 3001])
def test_lepton_single_step_scattered_states(gpu_tables, ora_tables, n):
    """One step from leptons scattered through an LP pulse (many events, every branch)."""
    b = I.random_states(n, seed=100 + n, gamma_range=(50.0, 6000.0), field_region=(-40.0, 10.0))
    f = Q.field(B.QED_FIELD_LP, a0=120.0, n_cycles=5.0, eta0=ETA0)
    for q in (-1, 1):
        gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, 1, q=q, dt=0.2, t0=10.0)
        compare_sets(gL.read(), oL.view(), 1e-12, "leptons")
        compare_sets(gG.read(), oG.view(), 1e-12, "photons", P_headless=True)
        assert c.events == oc.events and c.stored == oc.stored
        # |s|^2 can sit within rounding of 1: whether it is rescaled then changes s by ~1e-16 only
        assert abs(c.renormalised - oc.renormalised) <= 2 + oc.renormalised // 200
        assert c.status == 0


def test_lepton_many_steps_events(gpu_tables, ora_tables):
    b = I.random_states(1500, seed=5, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_CP, a0=80.0, n_cycles=5.0, eta0=ETA0)
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, 40, dt=0.1, t0=5.0)
    assert oc.events > 2000
    assert c.events == oc.events and c.chi_clamped == oc.chi_clamped
    compare_sets(gL.read(), oL.view(), 40e-12, "leptons")
    compare_sets(gG.read(), oG.view(), 40e-12, "photons", P_headless=True)


def test_headon_lp_trajectory(gpu_tables, ora_tables):
    """The 1e4-electron LP a0 = 50 collision (1 % spread, 1 mrad, random spins) on a 2000-electron
    subset, stepped through the whole pulse."""
    wl = I.HEADON_LP_SMALL
    b = wl.beam(n=2000)
    f = Q.laser_field(wl.laser)
    steps = 1300
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, steps, seed=wl.seed, dt=wl.dt)
    assert oc.events > 5000
    assert c.events == oc.events and c.stored == oc.stored
    tol = 1e-12 * steps
    compare_sets(gL.read(), oL.view(), tol, "leptons")
    compare_sets(gG.read(), oG.view(), tol, "photons", P_headless=True)


@pytest.mark.parametrize("flags", [
    B.QED_F_FULL & ~B.QED_F_TAU,                                         # per-step probability decision
    B.QED_F_FULL & ~(B.QED_F_SPIN_COLLAPSE | B.QED_F_POL_COLLAPSE),      # expectation values, no collapse
    B.QED_F_FULL & ~B.QED_F_RESOLVED,                                    # spin-averaged rates
    B.QED_F_FULL | B.QED_F_TBMT_PAPER,                                   # T-BMT as printed
    B.QED_F_FULL & ~(B.QED_F_SPIN_EVENT | B.QED_F_NONTRANSITION),
    B.QED_F_FULL & ~B.QED_F_RECOIL,
])
def test_lepton_modes(gpu_tables, ora_tables, flags):
    b = I.random_states(700, seed=flags % 1000, gamma_range=(100.0, 4000.0), field_region=(-30.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=100.0, n_cycles=4.0, eta0=ETA0)
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, 6, flags=flags, dt=0.15, t0=8.0)
    assert c.events == oc.events
    compare_sets(gL.read(), oL.view(), 6e-12, "leptons")
    compare_sets(gG.read(), oG.view(), 6e-12, "photons", P_headless=True)


def test_photon_store_threshold_and_empty(gpu_tables, ora_tables):
    b = I.random_states(300, seed=9, field_region=(-30.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=100.0, n_cycles=4.0, eta0=ETA0)
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, b, f, 5, dt=0.2, t0=8.0, store_min=2.0)
    assert c.below_store == oc.below_store and c.stored == oc.stored
    compare_sets(gG.read(), oG.view(), 5e-12, "photons", P_headless=True)
    # an empty buffer is a no-op
    e = {k: v[:0] for k, v in b.items()}
    gL, gG, oL, oG, c, oc = _run_lepton(gpu_tables, ora_tables, e, f, 2)
    assert gL.count() == 0 and gG.count() == 0 and c.events == 0 and c.status == 0


def test_nonfinite_particle_is_skipped_and_reported(gpu_tables, ora_tables):
    """A particle with a NaN is skipped and reported with its index (buffer overflow: test_gpu_overflow)."""
    b = I.random_states(400, seed=11, gamma_range=(1000.0, 5000.0), field_region=(-30.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=150.0, n_cycles=4.0, eta0=ETA0)
    bad = {k: v.copy() for k, v in b.items()}
    bad["mom"][17, 1] = np.nan
    g = gpu_particles(bad, FP64, -1, seed=3)
    ctr = Q.Counters()
    B.qed_push_step(gpu_tables.handle, f, Q.step_desc(0.1, 8.0, 0, 3), g.s, None, ctr.ptr)
    c = ctr.read()
    assert c.nonfinite == 1 and c.status == B.QED_ERR_NAN and c.first_bad == 17
    assert np.isnan(g.read()["mom"][17, 1])


def test_chi_above_table_is_clamped_and_counted(ora_tables):
    small = dict(DESC, chi_max=0.05, n_chi=8)
    gt = Q.Tables(**small)
    ot = O.tables(small["chi_min"], small["chi_max"], small["n_chi"], small["n_r"], small["y_lo"], small["y_hi"])
    b = I.random_states(500, seed=12, gamma_range=(2000.0, 5000.0), field_region=(-30.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=100.0, n_cycles=4.0, eta0=ETA0)
    gL, gG, oL, oG, c, oc = _run_lepton(gt, ot, b, f, 3, dt=0.2, t0=8.0)
    assert c.chi_clamped == oc.chi_clamped > 0
    compare_sets(gL.read(), oL.view(), 3e-12, "leptons")
    gt.close()


# ------------------------------------------------------------------------------------------------
# photon step, pairs, compaction
# ------------------------------------------------------------------------------------------------
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


@pytest.mark.parametrize("flags", [None, B.QED_F_FULL & ~B.QED_F_SPIN_COLLAPSE, B.QED_F_FULL & ~B.QED_F_TAU,
                                   B.QED_F_FULL | B.QED_F_BETA_BASIS,
                                   (B.QED_F_FULL & ~B.QED_F_SPIN_COLLAPSE) | B.QED_F_BETA_BASIS,
                                   B.QED_F_FULL | B.QED_F_REJECT])
def test_photon_steps_pairs_and_compaction(gpu_tables, ora_tables, flags):
    fl = B.QED_F_FULL if flags is None else flags
    b = _photon_inputs(2500, seed=21)
    f = Q.field(B.QED_FIELD_CP, a0=200.0, n_cycles=4.0, eta0=ETA0)
    of = as_oracle_field(f)
    gG = gpu_particles(b, FP64, B.QED_PHOTON, seed=4, photons=True)
    gE = Q.ParticleBuffer(5000, FP64, B.QED_ELECTRON)
    gP = Q.ParticleBuffer(5000, FP64, B.QED_POSITRON)
    ws = Q.CompactWorkspace(gG.capacity)
    oG = oracle_particles(b, seed=4)
    oE, oP = O.Particles(5000), O.Particles(5000)
    ctr, octr = Q.Counters(), O.Counters()
    steps = 25
    for s in range(steps):
        st = Q.step_desc(0.2, 6.0 + 0.2 * s, s, 4, fl)
        B.qed_pair_step(gpu_tables.handle, f, st, gG.s, gE.s, gP.s, ctr.ptr)
        B.qed_compact(gG.s, ws.ptr, ws.bytes)
        O.photon_step(ora_tables, of, as_oracle_step(st), oG, oE, oP, octr)
    torch.cuda.synchronize()
    c = ctr.read()
    assert octr.events > 100 and c.events == octr.events and c.status == 0
    tol = 1e-12 * steps
    compare_sets(gG.read(), oG.view(), tol, "photons")
    compare_sets(gE.read(), oE.view(), tol, "electrons")
    compare_sets(gP.read(), oP.view(), tol, "positrons")
    assert int(gG.n_dead.item()) == 0


def test_coupled_species_cascade_like(gpu_tables, ora_tables):
    """Electrons, their photons and the pairs those make, in two colliding CP pulses, with the
    'alive at step start' snapshot and compaction every step."""
    f = Q.field(B.QED_FIELD_CP_COUNTER, a0=300.0, n_cycles=3.0, phase=3 * math.pi - 4.0, eta0=I.eta0_for_wavelength(1.0))
    of = as_oracle_field(f)
    b = I.lepton_beam(300, 1000.0, direction=(1, 0, 0), z_range=(-0.5, 0.5), spin="random", seed=31)
    cap = 40000
    gE = Q.ParticleBuffer(cap, FP64, B.QED_ELECTRON, use_begin=True)
    gE.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    gE.init_tau(31)
    gPo = Q.ParticleBuffer(cap, FP64, B.QED_POSITRON, use_begin=True)
    gG = Q.ParticleBuffer(cap, FP64, B.QED_PHOTON, photons=True, use_begin=True)
    ws = Q.CompactWorkspace(cap)
    oE = oracle_particles(b, capacity=cap, seed=31)
    oPo, oG = O.Particles(cap), O.Particles(cap)
    ctr = Q.Counters()
    steps = 60
    for s in range(steps):
        st = Q.step_desc(0.1, 0.1 * s, s, 31, B.QED_F_FULL, photon_store_min=2.0)
        B.qed_snapshot_counts([gE.s, gPo.s, gG.s])
        B.qed_pair_step(gpu_tables.handle, f, st, gG.s, gE.s, gPo.s, ctr.ptr)
        B.qed_push_step(gpu_tables.handle, f, st, gE.s, gG.s, ctr.ptr)
        B.qed_push_step(gpu_tables.handle, f, st, gPo.s, gG.s, ctr.ptr)
        B.qed_compact(gG.s, ws.ptr, ws.bytes)
        oracle_full_step(ora_tables, of, as_oracle_step(st), [(oE, -1), (oPo, 1)], oG, oE, oPo)
    torch.cuda.synchronize()
    assert oPo.n > 0 and oG.n > 100
    tol = 1e-12 * steps
    compare_sets(gE.read(), oE.view(), tol, "electrons")
    compare_sets(gPo.read(), oPo.view(), tol, "positrons")
    compare_sets(gG.read(), oG.view(), tol, "photons", P_headless=True)
