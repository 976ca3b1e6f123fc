"""GPU parity of the table-free rejection sampler (QED_F_REJECT, Sec. 4.2) for emission against the FP64
oracle: FP64 path at 1e-12 per step with identical decisions and bound counts, FP32 path at 1e-5 per
step with fewer than 1e-5 decision flips per particle-step.  Pairs: the photon tests of the two parity
files carry the flag; the batched kernels: tests/test_gpu_batch.py."""
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
FLAGS = B.QED_F_FULL | B.QED_F_REJECT


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


def _run(gt, ot, b, f, steps, layout, q=-1, dt=0.1, t0=5.0, seed=7, cap_ph=400000):
    if layout == B.QED_FP64:
        gL = gpu_particles(b, layout, q, seed=seed)
        oL = oracle_particles(b, seed=seed)
    else:
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
        st = Q.step_desc(dt, t0 + s * dt, s, seed, FLAGS)
        B.qed_push_step(gt.handle, f, st, gL.s, gG.s, ctr.ptr)
        O.lepton_step(ot, of, as_oracle_step(st), q, oL, oG, octr)
    torch.cuda.synchronize()
    return gL, gG, oL, oG, ctr.read(), octr


@pytest.mark.parametrize("q", [-1, 1])
def test_fp64_rejection_lepton_steps(gpu_tables, ora_tables, q):
    b = I.random_states(1500, seed=61, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_CP, a0=80.0, n_cycles=5.0, eta0=ETA0)
    steps = 20
    gL, gG, oL, oG, c, oc = _run(gpu_tables, ora_tables, b, f, steps, B.QED_FP64, q=q)
    assert oc.events > 300 and c.events == oc.events and c.status == 0
    assert c.bound_exceeded == oc.bound_exceeded
    compare_sets(gL.read(), oL.view(), steps * 1e-12, "leptons")
    compare_sets(gG.read(), oG.view(), steps * 1e-12, "photons", P_headless=True)
    # the optical depth is not used in this mode: both sides keep their birth values (-ln u, equal but
    # for the last bit of the two logarithms)
    np.testing.assert_allclose(np.sort(gL.read()["tau"]), np.sort(oL.view()["tau"]), rtol=4e-16, atol=0)


def test_fp32_rejection_lepton_steps(gpu_tables, ora_tables):
    b = I.random_states(3000, seed=62, gamma_range=(200.0, 5000.0), field_region=(-35.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=120.0, n_cycles=5.0, eta0=ETA0)
    steps = 10
    flips, psteps = 0, 0
    for q in (-1, 1):
        gL, gG, oL, oG, c, oc = _run(gpu_tables, ora_tables, b, f, steps, B.QED_FP32, q=q, t0=10.0)
        assert oc.events > 300 and c.status == 0
        assert abs(int(c.bound_exceeded) - oc.bound_exceeded) <= max(2, 1e-3 * oc.bound_exceeded)
        f1, _ = compare_with_flips(gL.read(), oL.view(), steps * 1e-5, "leptons")
        f2, _ = compare_with_flips(gG.read(), oG.view(), steps * 1e-5, "photons", P_headless=True)
        flips += f1 + f2
        psteps += len(b["id"]) * steps
    assert flips <= max(1, 1e-5 * psteps), (flips, psteps)
