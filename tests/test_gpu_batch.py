"""The batched path (qed_batch_*: every instance and species in one persistent launch per time step,
the step counter on the device, CUDA-graph replay, autotuned launch shape).

* Against the single-buffer FP32 entry points (qed_snapshot_counts, qed_pair_step, qed_push_step,
  qed_compact per instance, with the same time and step per call): the same arithmetic and the same
  random draws, so every particle of every instance must agree bit for bit (sets matched by id, since
  appended daughters may sit in another order), and so must the event counters.
* Against the FP64 oracle on two instances (the FP32 bar of test_gpu_parity_fp32.py).
* The launch shape (kernel variant, blocks per SM, chunk, graph or direct launches) changes nothing.
* The autotuner picks a valid shape, records it in its cache and reuses it.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_08929_gb300 import binding as B
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import inputs as I

from parity_util import as_oracle_field, as_oracle_step, compare_with_flips, oracle_full_step

DESC = dict(chi_min=1e-3, chi_max=1e2, n_chi=24, n_r=256, y_lo=-20.0, y_hi=20.0)
FP32 = B.QED_FP32
DT, T0, STEP0 = 0.1, 0.25, 5


def test_batch_arguments_need_no_device():
    """Invalid handles and arguments are rejected before any CUDA call."""
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    lib = B.lib()
    import ctypes
    h = ctypes.c_void_p()
    d = B.QedBatchDesc()
    assert lib.qed_batch_create(None, None, 0, None, None, None) == B.QED_ERR_ARG
    assert lib.qed_batch_create(None, None, 1, ctypes.byref(d), None, ctypes.byref(h)) == B.QED_ERR_STATE
    assert lib.qed_batch_step(None, 1, None) == B.QED_ERR_STATE
    assert lib.qed_batch_set_tuning(None, None) == B.QED_ERR_STATE
    assert lib.qed_batch_tune(None, 1, None, None, None) == B.QED_ERR_STATE
    lib.qed_batch_destroy(None)


# ---- instances -------------------------------------------------------------------------------------
def _specs():
    """Five instances: uneven sizes (one empty, one single particle), LP / CP / counter-propagating CP,
    strong enough fields for emission and pair creation within a few steps."""
    e8, e1 = I.eta0_for_wavelength(0.8), I.eta0_for_wavelength(1.0)
    return [
        dict(n=3001, gamma=1500.0, field=Q.field(B.QED_FIELD_CP, a0=200.0, n_cycles=4.0, phase=4 * math.pi, eta0=e8),
             seed=11, spin_dir=(0.0, 0.0, 1.0), degree=1.0),
        dict(n=33, gamma=3000.0, field=Q.field(B.QED_FIELD_LP, a0=100.0, n_cycles=6.0, phase=6 * math.pi, eta0=e8),
             seed=12, spin_dir=(0.6, 0.0, 0.8), degree=0.5),
        dict(n=0, gamma=1000.0, field=Q.field(B.QED_FIELD_LP, a0=50.0, n_cycles=4.0, phase=4 * math.pi, eta0=e8),
             seed=13, spin_dir=(0.0, 1.0, 0.0), degree=0.0),
        dict(n=1, gamma=4000.0, field=Q.field(B.QED_FIELD_CP, a0=150.0, n_cycles=4.0, phase=4 * math.pi, eta0=e8),
             seed=14, spin_dir=(1.0, 0.0, 0.0), degree=1.0),
        dict(n=700, gamma=1000.0, field=Q.field(B.QED_FIELD_CP_COUNTER, a0=300.0, n_cycles=3.0,
                                                  phase=3 * math.pi - 4.0, eta0=e1),
             seed=15, spin_dir=(0.0, 0.0, -1.0), degree=0.3),
    ]


def _beam(k, sp):
    return I.lepton_beam(sp["n"], sp["gamma"], direction=(0.0, 0.0, -1.0), z_range=(-3.0, 3.0), transverse=2.0,
                         spin="degree", spin_dir=sp["spin_dir"], degree=sp["degree"], seed=100 + k,
                         id_offset=k << 40)


def _caps(sp):
    return (4 * sp["n"] + 2048, 4 * sp["n"] + 2048, 60 * sp["n"] + 4096)


def _load(bufs, k, sp):
    e = bufs[0]
    b = _beam(k, sp)
    e.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    if sp["n"]:
        e.init_tau(sp["seed"])


def _make_batch(tables, specs, tuning=None, flags=None):
    bt = Q.Batch(tables, [s["field"] for s in specs], [s["seed"] for s in specs], [_caps(s) for s in specs],
                 DT, t0=T0, step0=STEP0, flags=flags)
    for k, sp in enumerate(specs):
        _load(bt.buffers()[k], k, sp)
    if tuning is not None:
        bt.set_tuning(**tuning)
    return bt


def _single_path(tables, specs, steps, flags=None):
    """The same instances through the single-buffer entry points, one instance after another."""
    out, ctr = [], Q.Counters()
    for k, sp in enumerate(specs):
        ce, cp, cg = _caps(sp)
        e = Q.ParticleBuffer(ce, FP32, B.QED_ELECTRON, use_begin=True)
        p = Q.ParticleBuffer(cp, FP32, B.QED_POSITRON, use_begin=True)
        g = Q.ParticleBuffer(cg, FP32, B.QED_PHOTON, photons=True, use_begin=True)
        _load((e, p, g), k, sp)
        ws = Q.CompactWorkspace(cg)
        for s in range(steps):
            st = Q.step_desc(DT, T0 + float(s) * DT, STEP0 + s, sp["seed"], flags)
            B.qed_snapshot_counts([e.s, p.s, g.s])
            B.qed_pair_step(tables.handle, sp["field"], st, g.s, e.s, p.s, ctr.ptr)
            B.qed_push_step(tables.handle, sp["field"], st, e.s, g.s, ctr.ptr)
            B.qed_push_step(tables.handle, sp["field"], st, p.s, g.s, ctr.ptr)
            B.qed_compact(g.s, ws.ptr, ws.bytes)
        out.append((e, p, g))
    torch.cuda.synchronize()
    return out, ctr.read()


def _raw(buf):
    """(ids, raw float bits of the state rows), sorted by id."""
    n = buf.count()
    ids = buf.ids[:n].cpu().numpy()
    rows = buf.q[:, :n].permute(1, 0, 2).reshape(n, 12).contiguous().view(torch.int32).cpu().numpy()
    o = np.argsort(ids)
    return ids[o], rows[o]


def _assert_same(bufs_a, bufs_b, what):
    msgs = []
    for k, (A, Bb) in enumerate(zip(bufs_a, bufs_b)):
        for name, x, y in zip(("electrons", "positrons", "photons"), A, Bb):
            ia, ra = _raw(x)
            ib, rb = _raw(y)
            if not np.array_equal(ia, ib):
                msgs.append(f"instance {k} {name}: id sets differ ({len(ia)} vs {len(ib)})")
                continue
            bad = np.nonzero((ra != rb).any(axis=1))[0]
            if len(bad):
                fa, fb = ra[bad].view(np.float32), rb[bad].view(np.float32)
                rel = np.abs(fa - fb) / np.maximum(np.maximum(np.abs(fa), np.abs(fb)), 1e-30)
                msgs.append(f"instance {k} {name}: {len(bad)} of {len(ia)} rows differ, max rel by column "
                            f"{np.array2string(rel[:, :10].max(axis=0), precision=2)}")
    assert not msgs, what + ":\n" + "\n".join(msgs)


@pytest.fixture(scope="module")
def gpu_tables():
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    t = Q.Tables(**DESC)
    yield t
    t.close()


@pytest.mark.gpu
def test_batch_matches_single_buffer_path(gpu_tables):
    specs = _specs()
    steps = 30  # 7 graph launches of 4 steps, then 2 direct steps
    bt = _make_batch(gpu_tables, specs, dict(variant=0, blocks_per_sm=0, chunk=4, graph_steps=4))
    bt.step(steps)
    torch.cuda.synchronize()
    ref, rctr = _single_path(gpu_tables, specs, steps)
    c = bt.ctr.read()
    assert c.status == 0 and rctr.status == 0, (c.status, rctr.status)
    assert c.events > 1000 and sum(x[1].count() for x in ref) > 0, "no pairs: the test would not cover the photon step"
    _assert_same(bt.buffers(), ref, "batch vs single-buffer")
    for k in ("events", "stored", "dropped_capacity", "chi_clamped", "renormalised", "below_store", "nonfinite"):
        assert getattr(c, k) == getattr(rctr, k), (k, getattr(c, k), getattr(rctr, k))
    st = bt.stats()
    assert st.step == STEP0 + steps
    bt.close()


@pytest.mark.gpu
@pytest.mark.parametrize("flags", [B.QED_F_FULL | B.QED_F_TBMT_PAPER,
                                   B.QED_F_FULL & ~(B.QED_F_POL_COLLAPSE | B.QED_F_SPIN_COLLAPSE),
                                   B.QED_F_FULL | B.QED_F_AMM, B.QED_F_FULL | B.QED_F_LOOP,
                                   B.QED_F_FULL | B.QED_F_BETA_BASIS, B.QED_F_FULL | B.QED_F_REJECT])
def test_batch_matches_single_buffer_path_other_flags(gpu_tables, flags):
    """A flag set other than the full one runs the batched kernels that read the flags at run time."""
    specs = _specs()
    steps = 12
    bt = _make_batch(gpu_tables, specs, dict(variant=0, blocks_per_sm=0, chunk=4, graph_steps=4), flags=flags)
    bt.step(steps)
    torch.cuda.synchronize()
    ref, rctr = _single_path(gpu_tables, specs, steps, flags=flags)
    c = bt.ctr.read()
    assert c.status == 0 and rctr.status == 0, (c.status, rctr.status)
    assert c.events > 100
    _assert_same(bt.buffers(), ref, f"batch vs single-buffer, flags {flags:#x}")
    for k in ("events", "stored", "dropped_capacity", "renormalised", "below_store"):
        assert getattr(c, k) == getattr(rctr, k), (k, getattr(c, k), getattr(rctr, k))
    bt.close()


@pytest.mark.gpu
@pytest.mark.parametrize("tuning", [dict(variant=1, blocks_per_sm=1, chunk=1, graph_steps=0),
                                    dict(variant=2, blocks_per_sm=0, chunk=16, graph_steps=7),
                                    dict(variant=3, blocks_per_sm=0, chunk=3, graph_steps=1),
                                    dict(variant=4, blocks_per_sm=0, chunk=2, graph_steps=3)])
def test_batch_launch_shape_changes_nothing(gpu_tables, tuning):
    specs = _specs()
    steps = 16
    a = _make_batch(gpu_tables, specs, dict(variant=0, blocks_per_sm=0, chunk=4, graph_steps=0))
    b = _make_batch(gpu_tables, specs, tuning)
    a.step(steps)
    b.step(steps)
    torch.cuda.synchronize()
    ca, cb = a.ctr.read(), b.ctr.read()
    assert ca.events == cb.events and ca.stored == cb.stored and ca.renormalised == cb.renormalised
    _assert_same(a.buffers(), b.buffers(), f"shape {tuning}")
    sa, sb = a.stats(), b.stats()
    assert sa.particle_steps == sb.particle_steps and sa.step == sb.step == STEP0 + steps
    a.close()
    b.close()


@pytest.mark.gpu
def test_batch_particle_step_accounting(gpu_tables):
    specs = _specs()
    bt = _make_batch(gpu_tables, specs)
    total = 0
    for s in range(6):
        alive = sum(e.count() + p.count() + g.count() for e, p, g in bt.buffers())
        bt.step(1)
        torch.cuda.synchronize()
        total += alive
        st = bt.stats()
        assert st.particle_steps == total == sum(st.species_steps)
        assert sum(st.alive) == alive
    bt.close()


@pytest.mark.gpu
def test_batch_against_oracle():
    """Two instances of the batch against the FP64 oracle, stepped with the same times and draws."""
    desc = DESC
    gt = Q.Tables(**desc)
    ot = O.tables(*desc.values())
    specs = [_specs()[0], _specs()[4]]
    specs[0] = dict(specs[0], n=1500)
    bt = _make_batch(gt, specs)
    ora = []
    for (e, p, g), sp in zip(bt.buffers(), specs):
        r = e.read()
        cap = _caps(sp)
        oe = O.Particles.from_arrays(cap[0], r["pos"], r["mom"], r["spin"], r["w"], r["id"], tau=r["tau"])
        ora.append((oe, O.Particles(cap[1]), O.Particles(cap[2])))
    steps = 12
    bt.step(steps)
    for sp, (oe, op, og) in zip(specs, ora):
        of = as_oracle_field(sp["field"])
        for s in range(steps):
            st = Q.step_desc(DT, T0 + float(s) * DT, STEP0 + s, sp["seed"])
            oracle_full_step(ot, of, as_oracle_step(st), [(oe, -1), (op, 1)], og, oe, op)
    torch.cuda.synchronize()
    tol = 1e-5 * steps
    flips = 0
    for (e, p, g), (oe, op, og) in zip(bt.buffers(), ora):
        f1, _ = compare_with_flips(e.read(), oe.view(), tol, "electrons")
        f2, _ = compare_with_flips(p.read(), op.view(), tol, "positrons")
        f3, _ = compare_with_flips(g.read(), og.view(), tol, "photons", P_headless=True)
        flips += f1 + f2 + f3
    assert og.n > 100
    assert flips <= max(3, 1e-5 * steps * sum(len(x[2].read()["id"]) for x in bt.buffers()))
    bt.close()
    gt.close()


@pytest.mark.gpu
@pytest.mark.parametrize("graph_steps", [0, 5])
def test_kernel_events_time_every_step(gpu_tables, graph_steps):
    """Event pairs around the persistent kernel: recorded for every step, graph or direct, and the
    results stay those of a batch without them."""
    specs = _specs()
    steps = 5
    a = _make_batch(gpu_tables, specs, dict(variant=0, blocks_per_sm=0, chunk=4, graph_steps=graph_steps))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    a.set_kernel_events(ev)
    a.step(0)  # graph capture only (no step)
    assert a.stats().step == STEP0
    whole0, whole1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    whole0.record()
    a.step(steps)
    whole1.record()
    torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    assert all(m > 0 for m in ms) and sum(ms) <= whole0.elapsed_time(whole1) * 1.01
    b = _make_batch(gpu_tables, specs, dict(variant=0, blocks_per_sm=0, chunk=4, graph_steps=0))
    b.step(steps)
    torch.cuda.synchronize()
    _assert_same(a.buffers(), b.buffers(), "with kernel events")
    a.close()
    b.close()


@pytest.mark.gpu
def test_autotuner_picks_and_caches(gpu_tables, tmp_path):
    specs = _specs()
    bt = _make_batch(gpu_tables, specs)
    path = str(tmp_path / "tune.jsonl")
    s0 = bt.stats().step
    t1 = bt.tune(1, path)
    s1 = bt.stats().step
    assert s1 > s0  # the tuner's timed steps are real steps
    assert 0 <= t1.variant < 5 and t1.blocks_per_sm >= 1 and t1.chunk in (32, 64, 128) and t1.graph_steps == 8
    lines = open(path).read().strip().splitlines()
    assert len(lines) == 1 and '"variant": %d' % t1.variant in lines[0]
    t2 = bt.tune(1, path)  # cached: no timing, no steps
    assert bt.stats().step == s1
    assert (t2.variant, t2.blocks_per_sm, t2.chunk) == (t1.variant, t1.blocks_per_sm, t1.chunk)
    bt.step(3)
    torch.cuda.synchronize()
    assert bt.ctr.read().status == 0
    bt.close()
