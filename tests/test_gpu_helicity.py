"""The helicity-transfer analogues (Sec. 8.6.3, 8.6.4) through the batched FP32 path, both collisions as
instances of one batch, against the FP64 oracle stepping the same electrons with the same draws: at the
end of the crossing every particle within the n-step bar (n x 1e-5; fewer than 1e-5 flips per
particle-step), and the diagnostics (photons' circular polarization, positrons' longitudinal
polarization, per 1 GeV bin) equal within 0.02 wherever a bin holds more than 50 particles."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import diagnostics as D
from paper_2511_08929_gb300 import inputs as I

from parity_util import compare_with_flips, oracle_full_step

pytestmark = pytest.mark.gpu

DESC = dict(chi_min=1e-3, chi_max=1e2, n_chi=64, n_r=256, y_lo=-20.0, y_hi=20.0)
GEV = 1e9 / I.ME_EV


def test_helicity_batch_against_oracle():
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    n = 1500
    wls = [dataclasses.replace(I.HELICITY_LP_X14, n_electrons=n), dataclasses.replace(I.HELICITY_CP_X15, n_electrons=n)]
    gt = Q.Tables(**DESC)
    ot = O.tables(*DESC.values())
    fields = [Q.laser_field(w.laser) for w in wls]
    caps = [(30 * n, 30 * n, 120 * n)] * 2
    bt = Q.Batch(gt, fields, [w.seed for w in wls], caps, wls[0].dt, t0=0.0, step0=0)
    ora = []
    for k, (w, (e, p, g)) in enumerate(zip(wls, bt.buffers())):
        b = w.beam()
        b["id"] = b["id"] + np.uint64(k << 40)
        e.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
        e.init_tau(w.seed)
        r = e.read()
        ora.append([O.Particles.from_arrays(c, r["pos"], r["mom"], r["spin"], r["w"], r["id"], tau=r["tau"])
                    if i == 0 else O.Particles(c) for i, c in enumerate(caps[k])])
    steps = max(w.crossing_steps() for w in wls)
    bt.step(steps)
    for w, f, (oe, op, og) in zip(wls, fields, ora):
        of = O.field({"LP": O.FIELD_LP, "CP": O.FIELD_CP}[w.laser.kind], a0=w.laser.a0,
                     n_cycles=w.laser.n_cycles, eta0=w.laser.eta0)
        for s in range(steps):
            oracle_full_step(ot, of, O.step_desc(w.dt, s * w.dt, s, w.seed, O.F_FULL), [(oe, -1), (op, 1)], og, oe, op)
    torch.cuda.synchronize()
    assert bt.ctr.read().status == 0
    flips, psteps = 0, 0
    edges = [i * GEV for i in range(11)]
    for k, ((e, p, g), (oe, op, og)) in enumerate(zip(bt.buffers(), ora)):
        for buf, ob, name, ph in ((e, oe, "electrons", False), (p, op, "positrons", False), (g, og, "photons", True)):
            fl, _ = compare_with_flips(buf.read(), ob.view(), steps * 1e-5, name, P_headless=ph)
            flips += fl
            psteps += steps * max(buf.count(), 1)
        # the diagnostic of each analogue: the GPU's (computed on the device) against the oracle's
        buf, ob, photon = (g, og, True) if k == 0 else (p, op, False)
        d = D.polarization_vs_energy(buf, edges)
        v = ob.view()
        mom = v["mom"]
        pn = np.linalg.norm(mom, axis=1)
        en = pn if photon else np.sqrt(1.0 + pn * pn)
        comp = (v["spin"] * mom).sum(1) / pn
        idx = np.floor(en / GEV).astype(int)
        for i in range(10):
            sel = idx == i
            if sel.sum() > 50:
                assert d["count"][i] == pytest.approx(sel.sum(), rel=0.01, abs=2)
                assert abs(d["mean"][i] - comp[sel].mean()) < 0.02, (k, i, d["mean"][i], comp[sel].mean())
        top = [m for m, c in zip(d["mean"], d["count"]) if c > 20][-1]
        assert top > 0.6  # the analogue reproduces the helicity transfer on the GPU as well
    assert flips <= max(5, 1e-5 * psteps), (flips, psteps)
    bt.close()
    gt.close()
