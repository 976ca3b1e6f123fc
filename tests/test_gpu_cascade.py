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


AE = 7.2973525693e-3 / (2 * np.pi)


def _condition(st: dict, of, wl, t: float, dt: float, q: float) -> np.ndarray:
    """The condition number of each lepton's step: max(1, its T-BMT turn |Omega| dt, its field impulse
    dt (|E1| + |E2|) / |p|), with |E1|, |E2| the amplitudes of the two waves at the particle.  FP32 fields
    carry rounding relative to each wave's amplitude; a step whose impulse is several times the momentum,
    or that turns the spin by many radians, passes that rounding on multiplied (FP64 Boris push from the
    step's start, time-centred momentum, standard T-BMT vector)."""
    out = np.zeros(len(st["id"]))
    n2 = 2 * np.pi * wl.n_cycles

    def env(ph):
        return np.where((ph >= 0) & (ph <= n2), np.sin(ph / (2 * wl.n_cycles)) ** 2, 0.0)

    amp = wl.a0 * (env(t - st["pos"][:, 2]) + env(t + st["pos"][:, 2]))
    for i in range(len(st["id"])):
        E, B = (np.asarray(v) for v in O.field_eval(of, st["pos"][i], t))
        p = st["mom"][i]
        h = 0.5 * q * dt
        pm = p + h * E
        tv = h * B / np.sqrt(1 + pm @ pm)
        pl = pm + np.cross(pm + np.cross(pm, tv), 2 * tv / (1 + tv @ tv))
        pb = 0.5 * (p + pl + h * E)
        g = np.sqrt(1 + pb @ pb)
        b = pb / g
        Om = (AE + 1 / g) * B - (AE * g / (g + 1)) * (b @ B) * b - (AE + 1 / (g + 1)) * np.cross(b, E)
        out[i] = max(1.0, np.linalg.norm(Om) * dt, dt * amp[i] / max(np.linalg.norm(p), 1e-300))
    return out


@pytest.mark.gpu
def test_cascade_subset_against_oracle():
    """Five steps inside the cascade, each from the GPU's state.  Low-energy leptons at the nodes of the
    standing wave turn their spin by up to ~30 rad in one step (gamma ~ 6 in |B| ~ 900) and receive field
    impulses several times their momentum: such a step is ill-conditioned (a 1e-7 relative change of its
    inputs moves the spin by up to ~1e-5), so the bar of a lepton (and of the photon it emits) is
    1e-5 x its step's condition number (_condition); every other particle is held to 1e-5."""
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    wl = dataclasses.replace(I.CASCADE_2E8, n_electrons=4000, chunk=4000)
    gt = Q.Tables(**DESC)
    ot = O.tables(*DESC.values())
    f = Q.laser_field(wl.laser())
    of = as_oracle_field(f)
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
    flips, psteps, events, worst_turn = 0, 0, 0, 0.0
    for s in range(5):
        step = start + s
        pre = [x.read() for x in bufs]
        if s == 0:
            assert len(pre[1]["id"]) > 1000 and len(pre[2]["id"]) > 1000, [len(x["id"]) for x in pre]
        ora = [O.Particles.from_arrays(c, r["pos"], r["mom"], r["spin"], r["w"], r["id"], tau=r["tau"])
               for c, r in zip(caps, pre)]
        bt.step(1)
        st = Q.step_desc(wl.dt, float(step) * wl.dt, step, wl.seed, photon_store_min=wl.photon_store_min)
        ctr = oracle_full_step(ot, of, as_oracle_step(st), [(ora[0], -1), (ora[1], 1)], ora[2], ora[0], ora[1])
        torch.cuda.synchronize()
        events += ctr.events
        # each lepton's turn angle, and the same factor for the photon it emitted this step
        ids, fac = [], []
        for r, q in ((pre[0], -1.0), (pre[1], 1.0)):
            ang = _condition(r, of, wl, float(step) * wl.dt, wl.dt, q)
            worst_turn = max(worst_turn, float(ang.max(initial=0.0)))
            ids.append(r["id"])
            fac.append(ang)
            kids = np.array([O.child_ids(int(i), wl.seed, step)[0] for i in r["id"]], dtype=np.uint64)
            ids.append(kids)
            fac.append(ang)
        scale = (np.concatenate(ids), np.concatenate(fac))
        for buf, o, name, ph in zip(bufs, ora, ("electrons", "positrons", "photons"), (False, False, True)):
            fl, _ = compare_with_flips(buf.read(), o.view(), 1e-5, name, P_headless=ph, spin_scale=scale)
            flips += fl
        psteps += sum(len(x["id"]) for x in pre)
    assert bt.ctr.read().status == 0
    assert events > 1000 and worst_turn > 10.0
    assert flips <= max(3, 1e-5 * psteps), (flips, psteps)
    bt.close()
    gt.close()
