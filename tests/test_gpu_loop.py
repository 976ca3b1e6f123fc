"""GPU parity of the anomalous-moment switches against the oracle: QED_F_AMM (T-BMT with the
field-dependent a(chi), Sec. 8.6.2), QED_F_LOOP (g = 2 in T-BMT and the loop's Scorer term of App. A.1
in the no-emission update), QED_F_G2 (g = 2), and the a(chi) table they read.  Bars as for the default
flags: FP64 1e-12 per step, FP32 1e-5 per step with fewer than 1e-5 decision flips per particle-step."""
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
FLAGS = [B.QED_F_FULL | B.QED_F_AMM, B.QED_F_FULL | B.QED_F_LOOP, B.QED_F_FULL | B.QED_F_G2]


@pytest.fixture(scope="module")
def gpu_tables():
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    t = Q.Tables(**DESC)
    yield t
    t.close()


@pytest.fixture(scope="module")
def ora_tables():
    return O.tables(*DESC.values()).ensure_amm()


def test_amm_table_matches_oracle(gpu_tables, ora_tables):
    g = B.qed_tables_export_amm(gpu_tables.handle, gpu_tables.desc)
    np.testing.assert_allclose(g, ora_tables.amm, rtol=0, atol=1e-13)
    assert abs(math.exp(g[0]) / (7.2973525693e-3 / (2 * math.pi)) - 1) < 1e-4  # chi_min = 1e-3


def test_amm_lookup_matches_oracle(gpu_tables, ora_tables):
    rng = np.random.default_rng(4)
    n = 3000
    chi = np.concatenate([np.exp(rng.uniform(math.log(1e-5), math.log(1e3), n - 3)), [0.0, 1e-3, 1e2]])
    cd = torch.tensor(chi, device="cuda")
    rd = torch.full((n,), 0.5, dtype=torch.float64, device="cuda")
    ref = np.array([ora_tables.amm_lookup(c) for c in chi])
    for prec, tol in ((B.QED_FP64, 1e-13), (B.QED_FP32, 2e-6)):
        out = torch.zeros(B.QED_LOOKUP_COLS * n, dtype=torch.float64, device="cuda")
        B.qed_tables_lookup(gpu_tables.handle, prec, cd.data_ptr(), rd.data_ptr(), out.data_ptr(), n)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(n, -1)[:, 8]
        assert np.abs(got / ref - 1).max() <= tol, prec


def _lepton_run(gt, ot, b, f, steps, layout, flags, q=-1, dt=0.1, t0=5.0, seed=7, cap_ph=400000):
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


@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("q", [-1, 1])
def test_fp64_lepton_steps(gpu_tables, ora_tables, flags, q):
    """20 steps of leptons through a circular pulse at chi ~ 0.1-3, every branch taken."""
    b = I.random_states(1500, seed=31, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_CP, a0=80.0, n_cycles=5.0, eta0=ETA0)
    steps = 20
    gL, gG, oL, oG, c, oc = _lepton_run(gpu_tables, ora_tables, b, f, steps, B.QED_FP64, flags, q=q)
    assert oc.events > 500 and c.events == oc.events and c.status == 0
    compare_sets(gL.read(), oL.view(), steps * 1e-12, "leptons")
    compare_sets(gG.read(), oG.view(), steps * 1e-12, "photons", P_headless=True)


def test_switches_change_the_spin(gpu_tables):
    """The three switches act: on the same inputs each moves the spins away from the default run by
    far more than the parity bar (so the parity above is not vacuous)."""
    b = I.random_states(600, seed=32, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_CP, a0=80.0, n_cycles=5.0, eta0=ETA0)
    fl0 = B.QED_F_FULL & ~B.QED_F_EMIT  # classical spin motion only: no decision can differ
    base = None
    for fl in (fl0, fl0 | B.QED_F_AMM, fl0 | B.QED_F_G2):
        g = gpu_particles(b, B.QED_FP64, -1, seed=7)
        ctr = Q.Counters()
        for s in range(20):
            B.qed_push_step(gpu_tables.handle, f, Q.step_desc(0.1, 5.0 + 0.1 * s, s, 7, fl), g.s, None, ctr.ptr)
        torch.cuda.synchronize()
        sp = g.read()["spin"]
        if base is None:
            base = sp
        else:
            assert np.abs(sp - base).max() > 1e-6, fl


@pytest.mark.parametrize("flags", FLAGS)
def test_fp32_lepton_steps(gpu_tables, ora_tables, flags):
    b = I.random_states(3000, seed=33, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=120.0, n_cycles=5.0, eta0=ETA0)
    steps = 10
    flips, psteps = 0, 0
    for q in (-1, 1):
        gL, gG, oL, oG, c, oc = _lepton_run(gpu_tables, ora_tables, b, f, steps, B.QED_FP32, flags, q=q, t0=10.0)
        assert oc.events > 300 and c.status == 0
        f1, _ = compare_with_flips(gL.read(), oL.view(), steps * 1e-5, "leptons")
        f2, _ = compare_with_flips(gG.read(), oG.view(), steps * 1e-5, "photons", P_headless=True)
        flips += f1 + f2
        psteps += len(b["id"]) * steps
    assert flips <= max(1, 1e-5 * psteps), (flips, psteps)


def test_contradictory_switches_are_rejected(gpu_tables):
    b = I.random_states(4, seed=1)
    g = gpu_particles(b, B.QED_FP64, -1, seed=7)
    f = Q.field(B.QED_FIELD_CP, a0=10.0, n_cycles=2.0, eta0=ETA0)
    ctr = Q.Counters()
    for bad in (B.QED_F_AMM | B.QED_F_G2, B.QED_F_AMM | B.QED_F_LOOP):
        st = Q.step_desc(0.1, 0.0, 0, 1, B.QED_F_FULL | bad)
        with pytest.raises(B.QedError) as e:
            B.qed_push_step(gpu_tables.handle, f, st, g.s, None, ctr.ptr)
        assert e.value.status == -1  # QED_ERR_ARG
