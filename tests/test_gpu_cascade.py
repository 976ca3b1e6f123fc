"""The large-cascade workload (two colliding CP pulses, a0 = 500, electrons of gamma 1000 at the
collision point) on a subset of its electrons: the batched FP32 path is advanced into the cascade, its
three species are read back, and from that state the GPU and the FP64 oracle take the same steps (pair
creation, emission, compaction, the photon storage threshold), compared by id at the FP32 bar (n x 1e-5
per particle, fewer than 1e-5 decision flips per particle-step)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import inputs as I

from parity_util import as_oracle_field, as_oracle_step, compare_with_flips, oracle_full_step

DESC = dict(chi_min=1e-4, chi_max=1e3, n_chi=64, n_r=256, y_lo=-20.0, y_hi=20.0)


def test_workload_generator_chunks():
    """Chunks are independent and reproducible; the subset equals the beam's first chunk's head."""
    wl = dataclasses.replace(I.CASCADE_2E8, n_electrons=2500, chunk=1000)
    assert wl.n_chunks() == 3
    a, b = wl.chunk_beam(1), wl.chunk_beam(1)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    c2 = wl.chunk_beam(2)
    assert len(c2["id"]) == 500 and c2["id"][0] == 2001
    assert np.allclose(np.linalg.norm(a["mom"], axis=1), np.sqrt(1000.0 ** 2 - 1))
    assert np.all(a["mom"][:, 2] == 0) and np.all(np.abs(a["pos"][:, 2]) <= np.pi / 2)


@pytest.mark.gpu
def test_cascade_subset_against_oracle():
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    wl = dataclasses.replace(I.CASCADE_2E8, n_electrons=4000, chunk=4000)
    gt = Q.Tables(**DESC)
    ot = O.tables(*DESC.values())
    f = Q.laser_field(wl.laser())
    caps = (200000, 200000, 400000)
    bt = Q.Batch(gt, [f], [wl.seed], [caps], wl.dt, t0=0.0, step0=0, photon_store_min=wl.photon_store_min)
    e = bt.buffers()[0][0]
    b = wl.chunk_beam(0)
    e.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    e.init_tau(wl.seed)
    start = 900  # inside the cascade: pairs are being made
    bt.step(start)
    torch.cuda.synchronize()
    bufs = bt.buffers()[0]
    st0 = [x.read() for x in bufs]
    assert len(st0[1]["id"]) > 1000 and len(st0[2]["id"]) > 1000, [len(x["id"]) for x in st0]
    ora = [O.Particles.from_arrays(c, r["pos"], r["mom"], r["spin"], r["w"], r["id"], tau=r["tau"])
           for c, r in zip(caps, st0)]
    steps = 10
    bt.step(steps)
    of = as_oracle_field(f)
    ctr = O.Counters()
    for s in range(steps):
        st = Q.step_desc(wl.dt, float(start + s) * wl.dt, start + s, wl.seed, photon_store_min=wl.photon_store_min)
        oracle_full_step(ot, of, as_oracle_step(st), [(ora[0], -1), (ora[1], 1)], ora[2], ora[0], ora[1], ctr)
    torch.cuda.synchronize()
    assert bt.ctr.read().status == 0
    assert ctr.events > 500  # emissions and pairs in the window
    assert ora[1].n > len(st0[1]["id"])  # positrons were made
    tol = 1e-5 * steps
    flips = 0
    psteps = steps * sum(len(x["id"]) for x in st0)
    for buf, o, name, ph in zip(bufs, ora, ("electrons", "positrons", "photons"), (False, False, True)):
        fl, _ = compare_with_flips(buf.read(), o.view(), tol, name, P_headless=ph)
        flips += fl
    assert flips <= max(3, 1e-5 * psteps), (flips, psteps)
    bt.close()
    gt.close()
