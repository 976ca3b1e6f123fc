"""Buffer overflow on the GPU against the oracle (FP64 and FP32 single-buffer paths, the batched path).

When the daughters of a step do not all fit, the library applies the events whose daughters got a slot
and leaves the others unapplied: the parent keeps the state the classical part of its step gave it and
its spent optical depth (it tries again next step), a pair is stored whole or not at all, counts stop
at capacity, and every refused event is counted in dropped_capacity with status QED_ERR_CAPACITY.
Which events of an overflowing step get the last slots is not fixed by the method (the oracle takes
them in parent order, the device in reservation order), so each step is checked against two oracle
runs from the GPU's own state before the step: one with room for every daughter (A: every event
applied) and one with no room at all (B: every event refused).  On the GPU:

* exactly min(room, events asking) events got daughters, and each daughter equals the oracle's
  daughter of the same parent (matched by id, A);
* a parent whose daughters were stored equals its A state; a parent whose daughters were refused equals
  its B state; every other particle equals both;
* no electron is stored without its positron (the pair's two ids come from one parent);
* the counters: events applied, dropped = events asking - stored, status and first_bad (an index of a
  refused parent).
"""
import numpy as np
import pytest

import oracle as O
from paper_2511_08929_gb300 import binding as B
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import inputs as I

from parity_util import as_oracle_field, as_oracle_step, by_id, rel_vec

pytestmark = pytest.mark.gpu

ETA0 = I.eta0_for_wavelength(0.8)
DESC = dict(chi_min=1e-3, chi_max=1e2, n_chi=24, n_r=64, y_lo=-20.0, y_hi=20.0)
TOL = {B.QED_FP64: 1e-11, B.QED_FP32: 1e-5}


@pytest.fixture(scope="module")
def gpu_tables():
    t = Q.Tables(**DESC)
    yield t
    t.close()


@pytest.fixture(scope="module")
def ora_tables():
    return O.tables(*DESC.values())


def _oparts(d, cap=None):
    cap = max(len(d["id"]), 1) if cap is None else cap
    return O.Particles.from_arrays(cap, d["pos"], d["mom"], d["spin"], d["w"], d["id"], tau=d["tau"])


def _rows(d, ids):
    """The rows of state dict d with the given ids (in that order)."""
    pos = {int(i): k for k, i in enumerate(d["id"])}
    ix = np.array([pos[int(i)] for i in ids], dtype=np.int64)
    return {k: v[ix] for k, v in d.items()}


def _err(g, o, P_headless=False):
    """per-particle error of state g against o (same id order)"""
    e = np.maximum(rel_vec(g["pos"], o["pos"], 1.0), rel_vec(g["mom"], o["mom"], 1e-300))
    sg, so = g["spin"], o["spin"]
    if P_headless:
        k = o["mom"] / np.maximum(np.linalg.norm(o["mom"], axis=1, keepdims=True), 1e-300)
        gpar, opar = (sg * k).sum(1, keepdims=True) * k, (so * k).sum(1, keepdims=True) * k
        flip = ((sg - gpar) * (so - opar)).sum(1) < 0
        sg = np.where(flip[:, None], 2 * gpar - sg, sg)
    e = np.maximum(e, np.linalg.norm(sg - so, axis=1))
    fin = np.isfinite(o["tau"]) & np.isfinite(g["tau"])
    e = np.maximum(e, np.where(fin, np.abs(g["tau"] - o["tau"]) / np.maximum(np.abs(o["tau"]), 1.0), 0.0))
    return np.maximum(e, np.abs(g["w"] - o["w"]))


def _check_states(gpu, expected, tol, what, P_headless=False, flips_ok=0):
    """gpu and expected hold the same ids; rows beyond tol are decision flips (FP32 only)."""
    g, o = by_id(gpu), by_id(expected)
    assert np.array_equal(g["id"], o["id"]), f"{what}: id sets differ"
    e = _err(g, o, P_headless)
    bad = int((e > tol).sum())
    assert bad <= flips_ok, f"{what}: {bad} particles beyond {tol} (worst {e.max(initial=0):.3g})"
    return bad


def _child_photon_ids(ids, seed, step):
    return np.array([O.child_ids(int(i), seed, step)[0] for i in ids], dtype=np.uint64)


def _child_pair_ids(ids, seed, step):
    c = [O.child_ids(int(i), seed, step) for i in ids]
    return np.array([a for a, _ in c], dtype=np.uint64), np.array([b for _, b in c], dtype=np.uint64)


def _lepton_outcome(pre, gpu_after, gpu_new_ph, A_L, A_G, B_L, seed, step, room, tol, what, flips_ok):
    """Check one lepton step under a photon budget `room`; returns (asking, stored, refused parent ids)."""
    asking = A_G["id"]  # every photon the events would store (their parents' children)
    stored = gpu_new_ph["id"]
    assert len(stored) == min(room, len(asking)), f"{what}: stored {len(stored)} of {len(asking)}, room {room}"
    assert set(stored.tolist()) <= set(asking.tolist()), f"{what}: a stored photon the oracle does not emit"
    _check_states(gpu_new_ph, _rows(A_G, stored), tol, what + " photons", P_headless=True, flips_ok=flips_ok)
    kids = _child_photon_ids(pre["id"], seed, step)
    asked = np.isin(kids, asking)
    got = np.isin(kids, stored)
    refused_ids = pre["id"][asked & ~got]
    applied_ids = pre["id"][~(asked & ~got)]
    exp = {k: np.concatenate([_rows(A_L, applied_ids)[k], _rows(B_L, refused_ids)[k]]) for k in A_L}
    _check_states(gpu_after, exp, tol, what + " leptons", flips_ok=flips_ok)
    return len(asking), len(stored), refused_ids


def _photon_outcome(pre, gpu_surv, gpu_new_e, gpu_new_p, A_G, A_E, A_P, B_G, seed, step, room, tol, what, flips_ok):
    """Check one photon step (pairs) under a pair budget `room`; returns (asking, made, refused parent ids)."""
    asking = len(A_E["id"])
    made = len(gpu_new_e["id"])
    assert made == len(gpu_new_p["id"]), f"{what}: {made} electrons but {len(gpu_new_p['id'])} positrons"
    assert made == min(room, asking), f"{what}: {made} pairs of {asking}, room {room}"
    kid_e, kid_p = _child_pair_ids(pre["id"], seed, step)
    conv = np.isin(kid_e, gpu_new_e["id"])
    # the electron and positron of every stored pair come from the same photon
    assert np.array_equal(np.sort(kid_p[conv]), np.sort(gpu_new_p["id"])), f"{what}: pair halves from different photons"
    asked = np.isin(kid_e, A_E["id"])
    assert not np.any(conv & ~asked)
    _check_states(gpu_new_e, _rows(A_E, gpu_new_e["id"]), tol, what + " electrons", flips_ok=flips_ok)
    _check_states(gpu_new_p, _rows(A_P, gpu_new_p["id"]), tol, what + " positrons", flips_ok=flips_ok)
    survivors = pre["id"][~conv]
    assert set(gpu_surv["id"].tolist()) == set(survivors.tolist()), f"{what}: surviving photon set differs"
    _check_states(gpu_surv, _rows(B_G, survivors), tol, what + " photons", P_headless=True, flips_ok=flips_ok)
    return asking, made, pre["id"][asked & ~conv]


def _oracle_lepton_runs(tb, of, ost, q, pre):
    A_L, A_G = _oparts(pre, None), O.Particles(max(4 * len(pre["id"]), 1))
    O.lepton_step(tb, of, ost, q, A_L, A_G)
    B_L = _oparts(pre, None)
    O.lepton_step(tb, of, ost, q, B_L, O.Particles(0))
    return A_L.view(), A_G.view(), B_L.view()


def _oracle_photon_runs(tb, of, ost, pre):
    n = max(len(pre["id"]), 1)
    A_G, A_E, A_P = _oparts(pre, None), O.Particles(n), O.Particles(n)
    O.photon_step(tb, of, ost, A_G, A_E, A_P)
    B_G = _oparts(pre, None)
    O.photon_step(tb, of, ost, B_G, O.Particles(0), O.Particles(0))
    return A_G.view(), A_E.view(), A_P.view(), B_G.view()


# ------------------------------------------------------------------------------------------------
# single-buffer entry points
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("layout", [B.QED_FP64, B.QED_FP32])
def test_lepton_step_photon_overflow(gpu_tables, ora_tables, layout):
    b = I.random_states(2000, seed=31, gamma_range=(1000.0, 5000.0), field_region=(-30.0, 5.0))
    f = Q.field(B.QED_FIELD_LP, a0=150.0, n_cycles=4.0, eta0=ETA0)
    of = as_oracle_field(f)
    cap = 260
    gL = Q.ParticleBuffer(2000, layout, B.QED_ELECTRON)
    gL.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    gL.init_tau(3)
    gG = Q.ParticleBuffer(cap, layout, B.QED_PHOTON)
    ctr = Q.Counters()
    tol, flips = TOL[layout], (0 if layout == B.QED_FP64 else 1)
    tot_drop = 0
    for s in range(5):
        st = Q.step_desc(0.3, 8.0 + 0.3 * s, s, 3)
        pre, n0 = gL.read(), gG.count()
        c0 = ctr.read()
        B.qed_push_step(gpu_tables.handle, f, st, gL.s, gG.s, ctr.ptr)
        after, ph = gL.read(), gG.read()
        new = {k: v[n0:] for k, v in ph.items()}
        A_L, A_G, B_L = _oracle_lepton_runs(ora_tables, of, as_oracle_step(st), -1, pre)
        asking, stored, refused = _lepton_outcome(pre, after, new, A_L, A_G, B_L, 3, s, cap - n0, tol,
                                                  f"step {s}", flips)
        c = ctr.read()
        assert c.dropped_capacity - c0.dropped_capacity == asking - stored
        assert c.stored - c0.stored == stored
        assert gG.count() == n0 + stored <= cap
        if asking > stored:
            assert c.status == B.QED_ERR_CAPACITY
            assert int(pre["id"][c.first_bad]) in set(int(i) for i in refused) or c0.status != 0
        tot_drop += asking - stored
    assert tot_drop > 50 and gG.count() == cap  # the buffer filled and later events were refused


@pytest.mark.parametrize("layout", [B.QED_FP64, B.QED_FP32])
def test_pair_step_overflow_is_whole_pairs(gpu_tables, ora_tables, layout):
    """The positron buffer is the smaller one, the case that used to leave an electron without its
    positron: pairs are made while both have room, the rest leave their photon alive (state B)."""
    rng = np.random.default_rng(21)
    n = 1500
    d = np.column_stack([rng.normal(0, 0.05, n), rng.normal(0, 0.05, n), -np.ones(n)])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    e = 3000.0 * np.exp(rng.uniform(-1.0, 0.5, n))
    P = rng.normal(size=(n, 3))
    P *= rng.uniform(0, 1, (n, 1)) / np.linalg.norm(P, axis=1, keepdims=True)
    b = {"pos": np.column_stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-35, 5, n)]),
         "mom": d * e[:, None], "spin": P, "w": rng.uniform(0.5, 2, n), "id": np.arange(n, dtype=np.uint64) * 104729 + 1}
    f = Q.field(B.QED_FIELD_CP, a0=200.0, n_cycles=4.0, eta0=ETA0)
    of = as_oracle_field(f)
    gG = Q.ParticleBuffer(n, layout, B.QED_PHOTON, photons=True)
    gG.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"])
    gG.init_tau(4)
    cap_e, cap_p = 60, 35
    gE = Q.ParticleBuffer(cap_e, layout, B.QED_ELECTRON)
    gP = Q.ParticleBuffer(cap_p, layout, B.QED_POSITRON)
    ws = Q.CompactWorkspace(n)
    ctr = Q.Counters()
    tol, flips = TOL[layout], (0 if layout == B.QED_FP64 else 1)
    refused_total = 0
    for s in range(4):
        st = Q.step_desc(0.2, 10.0 + 0.2 * s, s, 4)
        pre, e0, p0 = gG.read(), gE.count(), gP.count()
        c0 = ctr.read()
        B.qed_pair_step(gpu_tables.handle, f, st, gG.s, gE.s, gP.s, ctr.ptr)
        B.qed_compact(gG.s, ws.ptr, ws.bytes)
        ev, pv = gE.read(), gP.read()
        new_e = {k: v[e0:] for k, v in ev.items()}
        new_p = {k: v[p0:] for k, v in pv.items()}
        A_G, A_E, A_P, B_G = _oracle_photon_runs(ora_tables, of, as_oracle_step(st), pre)
        asking, made, refused = _photon_outcome(pre, gG.read(), new_e, new_p, A_G, A_E, A_P, B_G, 4, s,
                                                min(cap_e - e0, cap_p - p0), tol, f"step {s}", flips)
        c = ctr.read()
        assert c.events - c0.events == made and c.stored - c0.stored == 2 * made
        assert c.dropped_capacity - c0.dropped_capacity == asking - made
        assert gE.count() - e0 == gP.count() - p0 == made
        if asking > made:
            assert c.status == B.QED_ERR_CAPACITY
        refused_total += asking - made
    assert gP.count() == cap_p and gE.count() == gP.count() < cap_e and refused_total > 10
    # no electron without its positron: every stored electron's parent also gave a stored positron
    assert len(set(gE.read()["id"].tolist())) == gE.count()


# ------------------------------------------------------------------------------------------------
# the batched path
# ------------------------------------------------------------------------------------------------
def test_batched_overflow_of_every_species(gpu_tables, ora_tables):
    """Two collisions whose photon, electron and positron buffers overflow within a few steps: each step
    of the batch (pairs from the photons alive at its start, photons from the leptons alive at its start,
    daughters into the room the buffers had when it began) against oracle runs A and B per instance."""
    fields = [Q.field(B.QED_FIELD_CP, a0=250.0, n_cycles=4.0, eta0=ETA0),
              Q.field(B.QED_FIELD_LP, a0=200.0, n_cycles=4.0, phase=2.0, eta0=ETA0)]
    seeds = [7, 8]
    beams = [I.random_states(900, seed=41, gamma_range=(2000.0, 6000.0), field_region=(-30.0, 5.0)),
             I.random_states(600, seed=42, gamma_range=(2000.0, 6000.0), field_region=(-30.0, 5.0))]
    beams[1]["id"] = beams[1]["id"] + (1 << 40)
    caps = [(1000, 6, 700), (700, 4, 500)]  # (electrons, positrons, photons)
    bt = Q.Batch(gpu_tables, fields, seeds, caps, 0.25, t0=8.0, step0=0)
    bt.set_tuning(variant=0, blocks_per_sm=0, chunk=4, graph_steps=0)
    for (e, p, g), bm, sd in zip(bt.buffers(), beams, seeds):
        e.load(bm["pos"], bm["mom"], bm["spin"], bm["w"], bm["id"])
        e.init_tau(sd)
    tol, flips = TOL[B.QED_FP32], 1
    full = {"e": False, "p": False, "g": False}
    for s in range(6):
        pres = [(e.read(), p.read(), g.read()) for e, p, g in bt.buffers()]
        c0 = bt.ctr.read()
        bt.step(1)
        c = bt.ctr.read()
        drop = stored_ph = made_pairs = 0
        for k, ((e, p, g), (pe, pp, pg)) in enumerate(zip(bt.buffers(), pres)):
            of = as_oracle_field(fields[k])
            ost = O.step_desc(0.25, 8.0 + 0.25 * s, s, seeds[k])
            ge, gp, gg = e.read(), p.read(), g.read()
            # pairs: photons alive at the step's start
            A_G, A_E, A_P, B_G = _oracle_photon_runs(ora_tables, of, ost, pg)
            new_e = _rows(ge, np.setdiff1d(ge["id"], pe["id"]))
            new_p = _rows(gp, np.setdiff1d(gp["id"], pp["id"]))
            kid_ph = _child_photon_ids(np.concatenate([pe["id"], pp["id"]]), seeds[k], s)
            surv_ids = np.setdiff1d(gg["id"], kid_ph)  # photons after the step that are not this step's children
            asking, made, _ = _photon_outcome(pg, _rows(gg, surv_ids), new_e, new_p, A_G, A_E, A_P, B_G, seeds[k], s,
                                              min(caps[k][0] - len(pe["id"]), caps[k][1] - len(pp["id"])), tol,
                                              f"instance {k} step {s} pairs", flips)
            drop += asking - made
            made_pairs += made
            # photons: the electrons and positrons alive at the step's start share the photon budget
            room = caps[k][2] - len(pg["id"])
            outs = []
            for pre, q in ((pe, -1), (pp, 1)):
                outs.append(_oracle_lepton_runs(ora_tables, of, ost, q, pre))
            A_Gall = {key: np.concatenate([o[1][key] for o in outs]) for key in outs[0][1]}
            new_ph = _rows(gg, np.intersect1d(gg["id"], kid_ph))
            asking_ph = len(A_Gall["id"])
            assert len(new_ph["id"]) == min(room, asking_ph), (k, s, len(new_ph["id"]), room, asking_ph)
            _check_states(new_ph, _rows(A_Gall, new_ph["id"]), tol, f"instance {k} step {s} photons", True, flips)
            for (pre, q), (A_L, _, B_L), after in zip(((pe, -1), (pp, 1)), outs, (ge, gp)):
                kids = _child_photon_ids(pre["id"], seeds[k], s)
                refused = np.isin(kids, A_Gall["id"]) & ~np.isin(kids, new_ph["id"])
                exp = {key: np.concatenate([_rows(A_L, pre["id"][~refused])[key], _rows(B_L, pre["id"][refused])[key]])
                       for key in A_L}
                _check_states(_rows(after, pre["id"]), exp, tol, f"instance {k} step {s} leptons {q}", flips_ok=flips)
            drop += asking_ph - len(new_ph["id"])
            stored_ph += len(new_ph["id"])
            full["e"] |= e.count() == caps[k][0]
            full["p"] |= p.count() == caps[k][1]
            full["g"] |= g.count() + made == caps[k][2]
            assert e.count() <= caps[k][0] and p.count() <= caps[k][1] and g.count() <= caps[k][2]
        assert c.dropped_capacity - c0.dropped_capacity == drop
        assert c.stored - c0.stored == stored_ph + 2 * made_pairs
        if drop:
            assert c.status == B.QED_ERR_CAPACITY
    assert full["p"] and full["g"], full
    bt.close()
