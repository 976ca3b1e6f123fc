"""qed_compact_noalloc (photon compaction on a fixed file-scope scratch, no allocation) against
qed_compact with a caller workspace: same survivors, bit for bit, over two calls in a row.

The file name keeps it last in collection, so it runs after every other test of a session as well as
on its own."""
import ctypes

import numpy as np
import pytest

from paper_2511_08929_gb300 import binding as B


def test_noalloc_rejects_capacity_above_limit():
    """The capacity check comes before any CUDA call, so it needs no device."""
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    lib = B.lib()
    s = B.QedParticles()
    s.layout, s.charge, s.capacity = B.QED_FP32, B.QED_PHOTON, B.QED_COMPACT_NOALLOC_MAX_CAPACITY + 1
    s.q0, s.q1, s.q2, s.id, s.count, s.dead, s.n_dead = 0x1000, 0x2000, 0x3000, 0x4000, 0x5000, 0x6000, 0x7000
    assert lib.qed_compact_noalloc(ctypes.byref(s), None) == B.QED_ERR_TOO_LARGE
    with pytest.raises(B.QedError, match="fixed scratch limit"):
        B.qed_compact_noalloc(s)
    lib.qed_status_string.restype = ctypes.c_char_p
    assert lib.qed_status_string(B.QED_ERR_TOO_LARGE) == b"size above the fixed limit of the call"
    assert lib.qed_compact_noalloc(None, None) == B.QED_ERR_ARG


def _fill(buf, n, rng):
    ids = rng.permutation(np.arange(1, n + 1, dtype=np.uint64) * 7919)
    buf.load(rng.normal(size=(n, 3)), rng.normal(size=(n, 3)) * 100.0, rng.uniform(-1, 1, (n, 3)) / 2,
             rng.uniform(0.5, 2.0, n), ids, tau=rng.exponential(size=n))
    return ids


def _raw(buf):
    """Raw state rows of [0, count) keyed by id (bit patterns, for an exact comparison)."""
    import torch
    n = buf.count()
    ids = buf.ids[:n].cpu().numpy()
    if buf.layout == B.QED_FP64:
        rows = buf.planes[:, :n].T.contiguous().view(torch.int64).cpu().numpy()
    else:
        rows = buf.q[:, :n].permute(1, 0, 2).reshape(n, 12).contiguous().view(torch.int32).cpu().numpy()
    order = np.argsort(ids)
    return ids[order], rows[order]


def _kill(buf, dead_ids):
    """Write the indices of dead_ids into buf's dead list, in a shuffled order."""
    import torch
    n = buf.count()
    ids = buf.ids[:n].cpu().numpy().view(np.uint64)
    where = {int(v): i for i, v in enumerate(ids)}
    idx = np.array([where[int(d)] for d in dead_ids], dtype=np.int64)
    np.random.default_rng(len(idx)).shuffle(idx)
    buf.dead[:len(idx)].copy_(torch.from_numpy(idx))
    buf.n_dead.fill_(len(idx))


@pytest.mark.gpu
@pytest.mark.parametrize("layout", [B.QED_FP32, B.QED_FP64])
@pytest.mark.parametrize("capacity,n", [(200003, 150001), (B.QED_COMPACT_NOALLOC_MAX_CAPACITY, 262144), (1000, 37)])
def test_noalloc_matches_workspace_compaction(layout, capacity, n):
    import torch
    from paper_2511_08929_gb300 import buffers as Q
    rng = np.random.default_rng(capacity + layout)
    ref = Q.ParticleBuffer(capacity, layout, B.QED_PHOTON, photons=True)
    out = Q.ParticleBuffer(capacity, layout, B.QED_PHOTON, photons=True)
    ids = _fill(ref, n, np.random.default_rng(7))
    _fill(out, n, np.random.default_rng(7))
    ws = Q.CompactWorkspace(capacity)
    alive = set(int(v) for v in ids)
    # two calls in a row: a scattered tenth, then a third plus the last twentieth of the array
    for frac, tail in ((0.1, False), (0.3, True)):
        m = ref.count()
        extra = ref.ids[m - m // 20 - 1:m].cpu().numpy().view(np.uint64) if tail else ()
        pool = np.array(sorted(alive), dtype=np.uint64)
        dead = set(int(v) for v in rng.choice(pool, int(frac * len(pool)), replace=False))
        dead |= set(int(v) for v in extra if int(v) in alive)
        dead = np.array(sorted(dead), dtype=np.uint64)
        _kill(ref, dead)
        _kill(out, dead)
        B.qed_compact(ref.s, ws.ptr, ws.bytes)
        B.qed_compact_noalloc(out.s)
        torch.cuda.synchronize()
        alive -= set(int(v) for v in dead)
        assert ref.count() == out.count() == len(alive)
        assert int(ref.n_dead.item()) == int(out.n_dead.item()) == 0
        ri, rr = _raw(ref)
        oi, orow = _raw(out)
        assert np.array_equal(ri, oi)
        assert set(int(v) for v in ri.view(np.uint64)) == alive
        assert np.array_equal(rr, orow)


@pytest.mark.gpu
def test_noalloc_calls_take_no_device_memory():
    """After the first call (the per-device scratch lookup), calls leave device memory untouched."""
    import torch
    from paper_2511_08929_gb300 import buffers as Q
    buf = Q.ParticleBuffer(50000, B.QED_FP32, B.QED_PHOTON, photons=True)
    _fill(buf, 40000, np.random.default_rng(3))
    B.qed_compact_noalloc(buf.s)
    torch.cuda.synchronize()
    dead = torch.arange(0, 40000, 4, dtype=torch.int64, device=buf.device)
    buf.dead[:len(dead)].copy_(dead)
    buf.n_dead.fill_(len(dead))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    held0 = torch.cuda.memory_reserved()
    B.qed_compact_noalloc(buf.s)
    B.qed_compact_noalloc(buf.s)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == held0
    assert buf.count() == 30000 and int(buf.n_dead.item()) == 0
