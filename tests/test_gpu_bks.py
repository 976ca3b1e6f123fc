"""GPU parity of the Sec. 8.3 variants against the oracle: spins resolved along +-beta
(QED_F_BETA_BASIS) and the magnetic field turning from z to y (QED_FIELD_ROT_B), on the FP64 path at
1e-12 per step and the FP32 path at 1e-5 per step (fewer than 1e-5 decision flips per particle-step).
The pair step with the beta basis is covered by the photon tests of the two parity files."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_08929_gb300 import binding as B
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import inputs as I

from parity_util import (as_oracle_field, as_oracle_step, compare_sets, compare_with_flips, gpu_particles,
                         oracle_particles)

pytestmark = pytest.mark.gpu

DESC = dict(chi_min=1e-3, chi_max=1e2, n_chi=24, n_r=256, y_lo=-20.0, y_hi=20.0)
ETA0 = I.eta0_for_wavelength(0.8)
GAMMA_1GEV = 1e9 / I.ME_EV


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


def _run(gt, ot, b, f, steps, layout, flags, q=-1, dt=0.1, t0=5.0, seed=7, cap_ph=400000):
    if layout == B.QED_FP64:
        gL = gpu_particles(b, layout, q, seed=seed)
        oL = oracle_particles(b, seed=seed)
    else:  # the oracle starts from the float-rounded state
        gL = Q.ParticleBuffer(len(b["id"]), layout, q)
        gL.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
        gL.init_tau(seed)
        r = gL.read()
        oL = O.Particles.from_arrays(len(b["id"]), r["pos"], r["mom"], r["spin"], r["w"], r["id"], tau=r["tau"])
    gG = Q.ParticleBuffer(cap_ph, layout, B.QED_PHOTON)
    oG = O.Particles(cap_ph)
    ctr, octr = Q.Counters(), O.Counters()
    of = as_oracle_field(f)
    for s in range(steps):
        st = Q.step_desc(dt, t0 + s * dt, s, seed, flags)
        B.qed_push_step(gt.handle, f, st, gL.s, gG.s, ctr.ptr)
        O.lepton_step(ot, of, as_oracle_step(st), q, oL, oG, octr)
    torch.cuda.synchronize()
    return gL, gG, oL, oG, ctr.read(), octr


BETA = [B.QED_F_FULL | B.QED_F_BETA_BASIS, (B.QED_F_FULL & ~B.QED_F_SPIN_COLLAPSE) | B.QED_F_BETA_BASIS]


@pytest.mark.parametrize("flags", BETA)
@pytest.mark.parametrize("q", [-1, 1])
def test_fp64_beta_basis_lepton_steps(gpu_tables, ora_tables, flags, q):
    b = I.random_states(1500, seed=51, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_CP, a0=80.0, n_cycles=5.0, eta0=ETA0)
    steps = 20
    gL, gG, oL, oG, c, oc = _run(gpu_tables, ora_tables, b, f, steps, B.QED_FP64, flags, q=q)
    assert oc.events > 500 and c.events == oc.events and c.status == 0
    compare_sets(gL.read(), oL.view(), steps * 1e-12, "leptons")
    compare_sets(gG.read(), oG.view(), steps * 1e-12, "photons", P_headless=True)


@pytest.mark.parametrize("flags", BETA)
def test_fp32_beta_basis_lepton_steps(gpu_tables, ora_tables, flags):
    b = I.random_states(3000, seed=52, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=120.0, n_cycles=5.0, eta0=ETA0)
    steps = 10
    flips, psteps = 0, 0
    for q in (-1, 1):
        gL, gG, oL, oG, c, oc = _run(gpu_tables, ora_tables, b, f, steps, B.QED_FP32, flags, q=q, t0=10.0)
        assert oc.events > 300 and c.status == 0
        f1, _ = compare_with_flips(gL.read(), oL.view(), steps * 1e-5, "leptons")
        f2, _ = compare_with_flips(gG.read(), oG.view(), steps * 1e-5, "photons", P_headless=True)
        flips += f1 + f2
        psteps += len(b["id"]) * steps
    assert flips <= max(1, 1e-5 * psteps), (flips, psteps)


def test_beta_basis_spins_end_on_beta(gpu_tables):
    """Every emitter's spin ends at +-beta: in a constant B along z an electron moving in the x-y plane
    has beta = -z, so with recoil and the push off every emitter's spin is (0, 0, +-1)."""
    n = 4000
    p = 3000.0
    f = Q.field(B.QED_FIELD_CONST, B0=(0, 0, 1.0 / (ETA0 * p)), eta0=ETA0)
    b = I.lepton_beam(n, math.sqrt(p * p + 1), direction=(1, 0, 0), spin="random", seed=53)
    fl = (B.QED_F_FULL & ~(B.QED_F_PUSH | B.QED_F_TBMT)) | B.QED_F_BETA_BASIS
    for layout in (B.QED_FP64, B.QED_FP32):
        g = gpu_particles(b, layout, -1, tau=np.full(n, 1e-9))
        ctr = Q.Counters()
        B.qed_push_step(gpu_tables.handle, f, Q.step_desc(0.05, 0.0, 0, 5, fl), g.s, None, ctr.ptr)
        torch.cuda.synchronize()
        s = g.read()["spin"]
        assert ctr.read().events == n
        tol = 1e-15 if layout == B.QED_FP64 else 1e-7
        np.testing.assert_allclose(np.abs(s[:, 2]), 1.0, atol=tol)
        np.testing.assert_allclose(s[:, :2], 0.0, atol=tol)


@pytest.mark.parametrize("layout", [B.QED_FP64, B.QED_FP32])
def test_rotating_field_steps(gpu_tables, ora_tables, layout):
    """1 GeV electrons through the turn of the rotating field (chi ~ 1 before it): parity over 60 steps
    that span the turn, every flag of the full set, both spin bases."""
    p = math.sqrt(GAMMA_1GEV ** 2 - 1)
    f = Q.field(B.QED_FIELD_ROT_B, n_cycles=0.5, phase=-2.0, B0=(0, 0, 1.0 / (ETA0 * p)), eta0=ETA0)
    b = I.lepton_beam(2000, GAMMA_1GEV, rel_spread=0.05, ang_sigma=0.1, direction=(1, 0, 0), spin="random",
                      seed=54)
    steps = 60
    for fl in (B.QED_F_FULL, B.QED_F_FULL | B.QED_F_BETA_BASIS):
        gL, gG, oL, oG, c, oc = _run(gpu_tables, ora_tables, b, f, steps, layout, fl, dt=0.1, t0=0.0)
        assert oc.events > 1000 and c.status == 0
        if layout == B.QED_FP64:
            assert c.events == oc.events
            compare_sets(gL.read(), oL.view(), steps * 1e-12, "leptons")
            compare_sets(gG.read(), oG.view(), steps * 1e-12, "photons", P_headless=True)
        else:
            f1, _ = compare_with_flips(gL.read(), oL.view(), steps * 1e-5, "leptons")
            f2, _ = compare_with_flips(gG.read(), oG.view(), steps * 1e-5, "photons", P_headless=True)
            assert f1 + f2 <= max(2, 1e-5 * 2000 * steps), (f1, f2)
    # the field did turn: B along y at the end of the run
    E, Bv = O.field_eval(as_oracle_field(f), np.zeros(3), steps * 0.1)
    assert abs(Bv[2]) < 1e-12 * abs(Bv[1])
