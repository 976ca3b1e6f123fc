"""The C ABI library builds for sm_103a and exports every entry point include/qed.h declares (CPU only:
nothing is called that needs a GPU)."""
import ctypes
import os
import subprocess

import pytest


def test_library_exports_every_declared_symbol():
    from paper_2511_08929_gb300 import build as bld
    from paper_2511_08929_gb300 import binding as B
    path = bld.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = B.declared_entry_points()
    assert "qed_push_step" in names and "qed_tables_build" in names and len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the ABI version and status strings need no device
    assert lib.qed_abi_version() == 3
    # qed_counters: eight 64-bit counters, status, pad, first_bad, and the call's reservation block
    assert ctypes.sizeof(B.QedCounters) == 9 * 8 + 8 + 8 + 4 * 8
    lib.qed_status_string.restype = ctypes.c_char_p
    assert lib.qed_status_string(-3) == b"particle buffer capacity exhausted"


def test_binding_flags_match_oracle_flags():
    """The oracle restates the physics switch bits independently; both must agree."""
    import oracle as O
    from paper_2511_08929_gb300 import binding as B
    pairs = {"TAU": O.F_TAU, "RECOIL": O.F_RECOIL, "SPIN_COLLAPSE": O.F_SPIN_COLLAPSE, "POL_COLLAPSE": O.F_POL_COLLAPSE,
             "NONTRANSITION": O.F_NONTRANSITION, "PUSH": O.F_PUSH, "TBMT": O.F_TBMT, "TBMT_PAPER": O.F_TBMT_PAPER,
             "EMIT": O.F_EMIT, "RESOLVED": O.F_RESOLVED, "MOVE": O.F_MOVE, "SPIN_EVENT": O.F_SPIN_EVENT,
             "POL_EVENT": O.F_POL_EVENT, "AMM": O.F_AMM, "LOOP": O.F_LOOP, "G2": O.F_G2,
             "BETA_BASIS": O.F_BETA_BASIS, "REJECT": O.F_REJECT}
    for k, v in pairs.items():
        assert getattr(B, "QED_F_" + k) == v, k
    assert B.QED_F_FULL == O.F_FULL


def test_argument_errors_need_no_device():
    """Null handles and pointers are rejected synchronously before any CUDA call."""
    from paper_2511_08929_gb300 import binding as B
    lib = B.lib()
    assert lib.qed_tables_build(None, None, None) == B.QED_ERR_ARG
    assert lib.qed_push_step(None, None, None, None, None, None, None) == B.QED_ERR_STATE
    assert lib.qed_counters_read(None, None, None) == B.QED_ERR_ARG
    assert lib.qed_compact_workspace_bytes(1000) >= 1000 * 17
    # the learned sampler on the batched step: a null batch is refused before any device work
    assert lib.qed_batch_set_mlp(None, None, 1e-4) == B.QED_ERR_STATE
    assert lib.qed_batch_mlp_last(None, 0, None, None, None, None, None, None, None) == B.QED_ERR_STATE
    assert lib.qed_mlp_sample(None, None, None, None, None, 0, 1e-4, 0, None, None, None, None, None) == B.QED_ERR_STATE
