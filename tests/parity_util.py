"""Helpers shared by the GPU parity tests: build both sides from the same seeded inputs, step them,
and compare particle sets matched by id."""
import numpy as np

import oracle as O
from paper_2511_08929_gb300 import binding as B
from paper_2511_08929_gb300 import buffers as Q


def oracle_particles(b, capacity=None, seed=None, tau=None):
    n = len(b["id"])
    p = O.Particles.from_arrays(capacity or max(n, 1), b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=tau)
    if seed is not None and tau is None:
        p.init_tau(seed)
    return p


def gpu_particles(b, layout, charge, capacity=None, seed=None, photons=False, tau=None):
    n = len(b["id"])
    g = Q.ParticleBuffer(capacity or max(n, 1), layout, charge, photons=photons)
    g.load(b["pos"], b["mom"], b["spin"], b["w"], b["id"], tau=tau)
    if seed is not None and tau is None:
        g.init_tau(seed)
    return g


def as_oracle_field(f: B.QedField):
    return O.field(f.kind, a0=f.a0, n_cycles=f.n_cycles, phase=f.phase, E0=tuple(f.E0), B0=tuple(f.B0), eta0=f.eta0)


def as_oracle_step(s: B.QedStepDesc):
    return O.step_desc(s.dt, s.t, s.step, s.seed, s.flags, s.photon_store_min, s.chi_floor)


def by_id(d):
    order = np.argsort(d["id"], kind="stable")
    return {k: v[order] for k, v in d.items()}


def rel_vec(a, b, floor):
    """per-row |a - b| / max(|a|, |b|, floor) for (n, 3) arrays"""
    num = np.linalg.norm(a - b, axis=1)
    den = np.maximum(np.maximum(np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)), floor)
    return num / den


def compare_sets(gpu: dict, ora: dict, rtol: float, what: str, P_headless: bool = False, pos_floor=1.0,
                 tau_finite_only=True):
    """Assert that the two particle sets hold the same ids and agree within rtol."""
    g, o = by_id(gpu), by_id(ora)
    assert len(g["id"]) == len(o["id"]), f"{what}: {len(g['id'])} gpu vs {len(o['id'])} oracle particles"
    assert np.array_equal(g["id"], o["id"]), f"{what}: id sets differ"
    worst = {}
    worst["pos"] = rel_vec(g["pos"], o["pos"], pos_floor).max(initial=0.0)
    worst["mom"] = rel_vec(g["mom"], o["mom"], 1e-300).max(initial=0.0)
    sg, so = g["spin"], o["spin"]
    if P_headless:  # P vectors are defined up to the sign of their transverse part: compare via k-parallel and outer part
        # flip the gpu vector where the transverse parts point opposite (P and -P_perp are the same state)
        k = o["mom"] / np.maximum(np.linalg.norm(o["mom"], axis=1, keepdims=True), 1e-300)
        gpar, opar = (sg * k).sum(1, keepdims=True) * k, (so * k).sum(1, keepdims=True) * k
        gperp, operp = sg - gpar, so - opar
        flip = (gperp * operp).sum(1) < 0
        sg = np.where(flip[:, None], gpar - gperp, sg)
    worst["spin"] = np.linalg.norm(sg - so, axis=1).max(initial=0.0)
    ft = np.isfinite(o["tau"]) if tau_finite_only else np.ones(len(o["tau"]), bool)
    assert np.array_equal(np.isfinite(g["tau"]), np.isfinite(o["tau"])), f"{what}: tau finiteness differs"
    worst["tau"] = (np.abs(g["tau"][ft] - o["tau"][ft]) / np.maximum(np.abs(o["tau"][ft]), 1.0)).max(initial=0.0)
    worst["w"] = np.abs(g["w"] - o["w"]).max(initial=0.0)
    bad = {k: v for k, v in worst.items() if not v <= rtol}
    assert not bad, f"{what}: beyond rtol {rtol}: {bad} (all: {worst})"
    return worst


def oracle_full_step(tb, f, st, leptons, photons, el=None, po=None, ctr=None):
    """One time step on the oracle with 'alive at step start' semantics: photons first (pairs are
    appended to the lepton buffers), then each lepton buffer over its particles present at the start."""
    ctr = ctr if ctr is not None else O.Counters()
    snaps = [(L, L.n) for (L, q) in leptons]
    if photons is not None and el is not None:
        O.photon_step(tb, f, st, photons, el, po, ctr)
    for (L, q), (_, n0) in zip(leptons, snaps):
        n_now = L.n
        L._s.n = n0
        O.lepton_step(tb, f, st, q, L, photons, ctr)
        L._s.n = n_now
    return ctr


def compare_with_flips(gpu: dict, ora: dict, rtol: float, what: str, P_headless: bool = False, pos_floor=1.0,
                       diverged=0.1, frac_ok=0.0, hard=None, spin_scale=None):
    """FP32-vs-FP64 comparison, matched by id.  A decision taken in FP32 next to its threshold (an event,
    a collapse sign) can go the other way: it leaves one daughter id on one side only and one on the
    other; such unmatched ids, and particles whose state moved apart by more than `diverged`, are flips.
    Every other particle must be within rtol, except that a fraction `frac_ok` of them may reach `hard`
    (ill-conditioned directions, see the FP32 tests).  spin_scale = (ids, factors >= 1): the momentum,
    spin (or P) and optical-depth bars of those particles are rtol x factor (a step whose own condition
    number is that factor; the optical depth depends on the turned spin through W(s.beta)).
    Returns (flipped decisions, error quantiles)."""
    g, o = by_id(gpu), by_id(ora)
    common, gi, oi = np.intersect1d(g["id"], o["id"], assume_unique=False, return_indices=True)
    only = (len(g["id"]) - len(common)) + (len(o["id"]) - len(common))
    gg = {k: v[gi] for k, v in g.items()}
    oo = {k: v[oi] for k, v in o.items()}
    e = {"pos": rel_vec(gg["pos"], oo["pos"], pos_floor), "mom": rel_vec(gg["mom"], oo["mom"], 1e-300)}
    sg, so = gg["spin"], oo["spin"]
    if P_headless:
        k = oo["mom"] / np.maximum(np.linalg.norm(oo["mom"], axis=1, keepdims=True), 1e-300)
        gpar, opar = (sg * k).sum(1, keepdims=True) * k, (so * k).sum(1, keepdims=True) * k
        gperp, operp = sg - gpar, so - opar
        flip = (gperp * operp).sum(1) < 0
        sg = np.where(flip[:, None], gpar - gperp, sg)
    e["spin"] = np.linalg.norm(sg - so, axis=1)
    if spin_scale is not None:
        sid, fac = np.asarray(spin_scale[0], dtype=np.uint64), np.asarray(spin_scale[1], dtype=np.float64)
        o_ = np.argsort(sid)
        sid, fac = sid[o_], fac[o_]
        ix = np.clip(np.searchsorted(sid, gg["id"]), 0, max(len(sid) - 1, 0))
        hit = (sid[ix] == gg["id"]) if len(sid) else np.zeros(len(gg["id"]), bool)
        div_ = np.where(hit, np.maximum(fac[ix] if len(sid) else 1.0, 1.0), 1.0)
        e["spin"] = e["spin"] / div_
        e["mom"] = e["mom"] / div_
    else:
        div_ = 1.0
    fin = np.isfinite(oo["tau"]) & np.isfinite(gg["tau"])
    e["tau"] = np.where(fin, np.abs(gg["tau"] - oo["tau"]) / np.maximum(np.abs(oo["tau"]), 1.0), 0.0) / div_
    e["w"] = np.abs(gg["w"] - oo["w"]) / np.maximum(np.abs(oo["w"]), 1e-300)
    worst_each = np.max(np.stack([e["pos"], e["mom"], e["spin"], e["tau"]]), axis=0)
    div = worst_each > diverged
    keep = ~div
    report = {}
    for k2, v in e.items():
        v = v[keep]
        report[k2] = {"max": float(v.max(initial=0.0)), "p999": float(np.quantile(v, 0.999)) if len(v) else 0.0,
                      "frac_above": float((v > rtol).mean()) if len(v) else 0.0}
    hard = rtol if hard is None else hard
    bad = {k2: r for k2, r in report.items() if r["max"] > hard or r["frac_above"] > frac_ok}
    assert not bad, f"{what}: beyond rtol {rtol} (hard {hard}, frac {frac_ok}): {bad}; {int(div.sum())} diverged, {only} unmatched"
    flips = int(div.sum()) + (only + 1) // 2
    return flips, report
