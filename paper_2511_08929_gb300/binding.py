"""ctypes binding of libqedgb (include/qed.h): the same entry points, argument marshalling only.

Every computation runs in the CUDA library.  If the library has not been built this module raises
instead of falling back to anything else.  Device memory is passed as integer addresses (e.g.
``tensor.data_ptr()``); streams as ``torch.cuda.Stream.cuda_stream`` integers (0 = default stream).
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqedgb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "qed.h")

QED_OK, QED_ERR_ARG, QED_ERR_CUDA, QED_ERR_CAPACITY, QED_ERR_RANGE, QED_ERR_NAN, QED_ERR_TIMEOUT, QED_ERR_STATE, \
    QED_ERR_NOMEM, QED_ERR_TOO_LARGE = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
QED_FP64, QED_FP32 = 0, 1
QED_ELECTRON, QED_PHOTON, QED_POSITRON = -1, 0, 1
QED_FIELD_CONST, QED_FIELD_LP, QED_FIELD_CP, QED_FIELD_CP_COUNTER, QED_FIELD_ROT_B = 0, 1, 2, 3, 4
QED_LOOKUP_COLS = 9
QED_COMPACT_NOALLOC_MAX_CAPACITY = int(re.search(r"#define QED_COMPACT_NOALLOC_MAX_CAPACITY (\d+)",
                                                 open(HEADER).read()).group(1))


def _flags_from_header():
    """Physics switch values, read from include/qed.h so the binding cannot drift from the ABI."""
    flags = {}
    txt = open(HEADER).read()
    for name, shift in re.findall(r"(QED_F_[A-Z0-9_]+) = 1u << (\d+)", txt):
        flags[name] = 1 << int(shift)
    return flags


_FLAGS = _flags_from_header()
globals().update(_FLAGS)
QED_F_FULL = (QED_F_TAU | QED_F_RECOIL | QED_F_SPIN_COLLAPSE | QED_F_POL_COLLAPSE | QED_F_NONTRANSITION  # noqa: F821
              | QED_F_PUSH | QED_F_TBMT | QED_F_EMIT | QED_F_RESOLVED | QED_F_MOVE | QED_F_SPIN_EVENT  # noqa: F821
              | QED_F_POL_EVENT)  # noqa: F821


class QedError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class QedTableDesc(C.Structure):
    _fields_ = [("chi_min", C.c_double), ("chi_max", C.c_double), ("n_chi", C.c_int32), ("n_r", C.c_int32),
                ("y_lo", C.c_double), ("y_hi", C.c_double)]


class QedField(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("a0", C.c_double), ("n_cycles", C.c_double),
                ("phase", C.c_double), ("E0", C.c_double * 3), ("B0", C.c_double * 3), ("eta0", C.c_double)]


class QedParticles(C.Structure):
    _fields_ = [("layout", C.c_int32), ("charge", C.c_int32), ("capacity", C.c_int64), ("count", C.c_void_p),
                ("begin", C.c_void_p)] + [(n, C.c_void_p) for n in
                                          ("x", "y", "z", "px", "py", "pz", "sx", "sy", "sz", "tau", "w",
                                           "q0", "q1", "q2", "id", "dead", "n_dead")]


class QedStepDesc(C.Structure):
    _fields_ = [("dt", C.c_double), ("t", C.c_double), ("step", C.c_uint64), ("seed", C.c_uint64),
                ("flags", C.c_uint32), ("pad", C.c_uint32), ("photon_store_min", C.c_double),
                ("chi_floor", C.c_double)]


class QedInstance(C.Structure):
    _fields_ = [("field", QedField), ("seed", C.c_uint64), ("electrons", QedParticles), ("positrons", QedParticles),
                ("photons", QedParticles)]


class QedBatchDesc(C.Structure):
    _fields_ = [("dt", C.c_double), ("t0", C.c_double), ("step0", C.c_uint64), ("flags", C.c_uint32),
                ("pad", C.c_int32), ("photon_store_min", C.c_double), ("chi_floor", C.c_double)]


class QedBatchTuning(C.Structure):
    _fields_ = [("variant", C.c_int32), ("blocks_per_sm", C.c_int32), ("chunk", C.c_int32), ("graph_steps", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class QedBatchStats(C.Structure):
    _fields_ = [("step", C.c_uint64), ("particle_steps", C.c_uint64), ("species_steps", C.c_uint64 * 3),
                ("alive", C.c_int64 * 3)]


class QedCounters(C.Structure):
    _fields_ = [("events", C.c_ulonglong), ("stored", C.c_ulonglong), ("dropped_capacity", C.c_ulonglong),
                ("chi_clamped", C.c_ulonglong), ("renormalised", C.c_ulonglong), ("below_store", C.c_ulonglong),
                ("nonfinite", C.c_ulonglong), ("rate_steps", C.c_ulonglong), ("bound_exceeded", C.c_ulonglong),
                ("status", C.c_int32),
                ("pad", C.c_int32), ("first_bad", C.c_int64),
                ("append_base", C.c_int64 * 2), ("append_budget", C.c_int64), ("append_next", C.c_ulonglong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad" and not k.startswith("append")}


_lock = threading.Lock()
_lib = None


def lib():
    """Load libqedgb.so (built in-tree by ``paper_2511_08929_gb300.build``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64, P = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.POINTER
            sig = {
                "qed_abi_version": (i32, []),
                "qed_status_string": (C.c_char_p, [i32]),
                "qed_tables_build": (i32, [P(QedTableDesc), P(vp), vp]),
                "qed_tables_export": (i32, [vp, vp, vp, vp, vp]),
                "qed_tables_export_amm": (i32, [vp, vp]),
                "qed_tables_destroy": (i32, [vp]),
                "qed_bessel_eval": (i32, [vp, i32, vp, vp, i64, vp]),
                "qed_tables_lookup": (i32, [vp, i32, vp, vp, vp, i64, vp]),
                "qed_init_tau": (i32, [P(QedParticles), u64, i64, vp]),
                "qed_push_step": (i32, [vp, P(QedField), P(QedStepDesc), P(QedParticles), P(QedParticles), vp, vp]),
                "qed_pair_step": (i32, [vp, P(QedField), P(QedStepDesc), P(QedParticles), P(QedParticles),
                                        P(QedParticles), vp, vp]),
                "qed_compact": (i32, [P(QedParticles), vp, C.c_size_t, vp]),
                "qed_compact_workspace_bytes": (C.c_size_t, [i64]),
                "qed_compact_noalloc": (i32, [P(QedParticles), vp]),
                "qed_snapshot_counts": (i32, [P(P(QedParticles)), i32, vp]),
                "qed_counters_read": (i32, [vp, P(QedCounters), vp]),
                "qed_batch_create": (i32, [vp, P(QedInstance), i32, P(QedBatchDesc), vp, P(vp)]),
                "qed_batch_set_tuning": (i32, [vp, P(QedBatchTuning)]),
                "qed_batch_get_tuning": (i32, [vp, P(QedBatchTuning)]),
                "qed_batch_step": (i32, [vp, i32, vp]),
                "qed_batch_set_kernel_events": (i32, [vp, P(vp), i32]),
                "qed_batch_tune": (i32, [vp, i32, C.c_char_p, P(QedBatchTuning), vp]),
                "qed_batch_stats_read": (i32, [vp, P(QedBatchStats), vp]),
                "qed_batch_destroy": (None, [vp]),
                "qed_mlp_create": (i32, [i64, vp, P(vp)]),
                "qed_mlp_destroy": (None, [vp]),
                "qed_mlp_get_params": (i32, [vp, vp]),
                "qed_mlp_set_params": (i32, [vp, vp]),
                "qed_mlp_targets": (i32, [vp, i64, u64, i64, vp, vp, vp, vp]),
                "qed_mlp_grad": (i32, [vp, vp, vp, i64, vp, vp, vp]),
                "qed_mlp_adamw": (i32, [vp, vp, C.c_float, C.c_float, vp]),
                "qed_mlp_train": (i32, [vp, vp, i64, i64, u64, i64, C.c_float, C.c_float, C.c_float, vp, vp]),
                "qed_mlp_forward": (i32, [vp, vp, i64, vp, vp]),
                "qed_mlp_sample": (i32, [vp, vp, vp, vp, vp, i64, C.c_double, i32, vp, vp, vp, vp, vp]),
                "qed_batch_set_mlp": (i32, [vp, vp, C.c_double]),
                "qed_batch_mlp_last": (i32, [vp, i64, vp, vp, vp, vp, vp, P(i64), P(C.c_ulonglong)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != QED_OK:
        raise QedError(status, where)


def status_string(status: int) -> str:
    try:
        return lib().qed_status_string(int(status)).decode()
    except RuntimeError:
        return str(status)


def qed_abi_version() -> int:
    return lib().qed_abi_version()


def qed_tables_build(desc: QedTableDesc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().qed_tables_build(C.byref(desc), C.byref(h), stream or None), "qed_tables_build")
    return h.value


def qed_tables_export(handle: int, desc: QedTableDesc):
    nc, nr = desc.n_chi, desc.n_r
    out = {"nlc_rate": np.zeros((2, nc)), "nbw_rate": np.zeros((2, nc)), "nlc_icdf": np.zeros((2, nc, nr)),
           "nbw_icdf": np.zeros((2, nc, nr))}
    ptr = [out[k].ctypes.data for k in ("nlc_rate", "nbw_rate", "nlc_icdf", "nbw_icdf")]
    _check(lib().qed_tables_export(handle, *ptr), "qed_tables_export")
    return out


def qed_tables_export_amm(handle: int, desc: QedTableDesc):
    """ln a(chi_i) on the rate grid, double[n_chi]."""
    out = np.zeros(desc.n_chi)
    _check(lib().qed_tables_export_amm(handle, out.ctypes.data), "qed_tables_export_amm")
    return out


def qed_tables_destroy(handle: int):
    _check(lib().qed_tables_destroy(handle), "qed_tables_destroy")


def qed_bessel_eval(handle: int, precision: int, x_dev: int, out_dev: int, n: int, stream: int = 0):
    _check(lib().qed_bessel_eval(handle, precision, x_dev, out_dev, n, stream or None), "qed_bessel_eval")


def qed_tables_lookup(handle: int, precision: int, chi_dev: int, r_dev: int, out_dev: int, n: int, stream: int = 0):
    _check(lib().qed_tables_lookup(handle, precision, chi_dev, r_dev, out_dev, n, stream or None), "qed_tables_lookup")


def qed_init_tau(p: QedParticles, seed: int, begin: int = 0, stream: int = 0):
    _check(lib().qed_init_tau(C.byref(p), seed, begin, stream or None), "qed_init_tau")


def qed_push_step(handle: int, field: QedField, step: QedStepDesc, leptons: QedParticles,
                  photons: QedParticles | None, counters_dev: int, stream: int = 0):
    _check(lib().qed_push_step(handle, C.byref(field), C.byref(step), C.byref(leptons),
                               C.byref(photons) if photons is not None else None, counters_dev, stream or None),
           "qed_push_step")


def qed_pair_step(handle: int, field: QedField, step: QedStepDesc, photons: QedParticles,
                  electrons: QedParticles | None, positrons: QedParticles | None, counters_dev: int,
                  stream: int = 0):
    _check(lib().qed_pair_step(handle, C.byref(field), C.byref(step), C.byref(photons),
                               C.byref(electrons) if electrons is not None else None,
                               C.byref(positrons) if positrons is not None else None, counters_dev, stream or None),
           "qed_pair_step")


def qed_compact_workspace_bytes(capacity: int) -> int:
    return lib().qed_compact_workspace_bytes(capacity)


def qed_compact(photons: QedParticles, workspace_dev: int, workspace_bytes: int, stream: int = 0):
    _check(lib().qed_compact(C.byref(photons), workspace_dev, workspace_bytes, stream or None), "qed_compact")


def qed_compact_noalloc(photons: QedParticles, stream: int = 0):
    st = lib().qed_compact_noalloc(C.byref(photons), stream or None)
    if st == QED_ERR_TOO_LARGE:
        raise QedError(st, f"qed_compact_noalloc: capacity {photons.capacity} is above the fixed scratch limit "
                           f"of {QED_COMPACT_NOALLOC_MAX_CAPACITY} photons (use qed_compact with a workspace)")
    _check(st, "qed_compact_noalloc")


def qed_snapshot_counts(buffers, stream: int = 0):
    arr = (C.POINTER(QedParticles) * len(buffers))(*[C.pointer(b) for b in buffers])
    _check(lib().qed_snapshot_counts(arr, len(buffers), stream or None), "qed_snapshot_counts")


def qed_counters_read(counters_dev: int, stream: int = 0) -> QedCounters:
    out = QedCounters()
    _check(lib().qed_counters_read(counters_dev, C.byref(out), stream or None), "qed_counters_read")
    return out


def qed_batch_create(tables, instances, desc: QedBatchDesc, counters_dev: int) -> int:
    """instances: a sequence of QedInstance; returns the batch handle."""
    arr = (QedInstance * len(instances))(*instances)
    h = C.c_void_p()
    _check(lib().qed_batch_create(tables, arr, len(instances), C.byref(desc), counters_dev, C.byref(h)),
           "qed_batch_create")
    return h.value


def qed_batch_set_tuning(batch: int, tuning: QedBatchTuning):
    _check(lib().qed_batch_set_tuning(batch, C.byref(tuning)), "qed_batch_set_tuning")


def qed_batch_get_tuning(batch: int) -> QedBatchTuning:
    out = QedBatchTuning()
    _check(lib().qed_batch_get_tuning(batch, C.byref(out)), "qed_batch_get_tuning")
    return out


def qed_batch_step(batch: int, n_steps: int, stream: int = 0):
    _check(lib().qed_batch_step(batch, n_steps, stream or None), "qed_batch_step")


def qed_batch_set_kernel_events(batch: int, events, n_pairs: int):
    """events: sequence of 2 n_pairs cudaEvent_t handles (integers, e.g. torch.cuda.Event.cuda_event)."""
    arr = (C.c_void_p * max(1, len(events)))(*events) if events else None
    _check(lib().qed_batch_set_kernel_events(batch, arr, n_pairs), "qed_batch_set_kernel_events")


def qed_batch_tune(batch: int, steps_per_candidate: int = 2, cache_path=None, stream: int = 0) -> QedBatchTuning:
    out = QedBatchTuning()
    path = cache_path.encode() if cache_path else None
    _check(lib().qed_batch_tune(batch, steps_per_candidate, path, C.byref(out), stream or None), "qed_batch_tune")
    return out


def qed_batch_stats_read(batch: int, stream: int = 0) -> QedBatchStats:
    out = QedBatchStats()
    _check(lib().qed_batch_stats_read(batch, C.byref(out), stream or None), "qed_batch_stats_read")
    return out


def qed_batch_destroy(batch: int):
    if batch:
        lib().qed_batch_destroy(batch)


QED_MLP_PARAMS = int(re.search(r"#define QED_MLP_PARAMS (\d+)", open(HEADER).read()).group(1))
QED_MLP_ALWAYS_TABLE = 1
QED_MLP_BRANCH_TABLE = 2


def qed_mlp_create(max_batch: int, init_params) -> int:
    """init_params: float32 numpy array of QED_MLP_PARAMS values."""
    a = np.ascontiguousarray(init_params, dtype=np.float32)
    if a.size != QED_MLP_PARAMS:
        raise ValueError(f"expected {QED_MLP_PARAMS} parameters, got {a.size}")
    h = C.c_void_p()
    _check(lib().qed_mlp_create(max_batch, a.ctypes.data, C.byref(h)), "qed_mlp_create")
    return h.value


def qed_mlp_destroy(m: int):
    if m:
        lib().qed_mlp_destroy(m)


def qed_mlp_get_params(m: int) -> np.ndarray:
    out = np.empty(QED_MLP_PARAMS, dtype=np.float32)
    _check(lib().qed_mlp_get_params(m, out.ctypes.data), "qed_mlp_get_params")
    return out


def qed_mlp_set_params(m: int, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != QED_MLP_PARAMS:
        raise ValueError(f"expected {QED_MLP_PARAMS} parameters, got {a.size}")
    _check(lib().qed_mlp_set_params(m, a.ctypes.data), "qed_mlp_set_params")


def qed_mlp_targets(tables: int, n: int, seed: int, first_index: int, x_dev: int, y_dev: int, raw_dev: int = 0,
                    stream: int = 0):
    _check(lib().qed_mlp_targets(tables, n, seed, first_index, x_dev, y_dev, raw_dev or None, stream or None),
           "qed_mlp_targets")


def qed_mlp_grad(m: int, x_dev: int, y_dev: int, n: int, grad_dev: int, loss_dev: int = 0, stream: int = 0):
    _check(lib().qed_mlp_grad(m, x_dev, y_dev, n, grad_dev, loss_dev or None, stream or None), "qed_mlp_grad")


def qed_mlp_adamw(m: int, grad_dev: int, lr: float, weight_decay: float, stream: int = 0):
    _check(lib().qed_mlp_adamw(m, grad_dev, lr, weight_decay, stream or None), "qed_mlp_adamw")


def qed_mlp_train(m: int, tables: int, steps: int, batch: int, seed: int, first_index: int, lr: float,
                  lr_final: float, weight_decay: float, loss_dev: int = 0, stream: int = 0):
    _check(lib().qed_mlp_train(m, tables, steps, batch, seed, first_index, lr, lr_final, weight_decay,
                               loss_dev or None, stream or None), "qed_mlp_train")


def qed_mlp_forward(m: int, x_dev: int, n: int, out_dev: int, stream: int = 0):
    _check(lib().qed_mlp_forward(m, x_dev, n, out_dev, stream or None), "qed_mlp_forward")


def qed_mlp_sample(m: int, tables: int, chi_dev: int, r_dev: int, s_dev: int, n: int, tol: float, flags: int,
                   out_dev: int, fell_dev: int = 0, n_fallback_dev: int = 0, stream: int = 0, err_dev: int = 0):
    _check(lib().qed_mlp_sample(m, tables, chi_dev, r_dev, s_dev, n, tol, flags, out_dev, fell_dev or None,
                                err_dev or None, n_fallback_dev or None, stream or None), "qed_mlp_sample")


def declared_entry_points():
    """Names of the functions include/qed.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qed_[a-z0-9_]+)\s*\(", txt)))


def qed_batch_set_mlp(batch: int, m: int, tol: float):
    """m = 0 (None) restores the tables on the batch's event path."""
    _check(lib().qed_batch_set_mlp(batch, m or None, tol), "qed_batch_set_mlp")


def qed_batch_mlp_last(batch: int, n_max: int):
    """The last step's sampler inputs and outputs of its first n_max events: (n_events, n_fallback_total,
    dict of chi, r, s_beta (float64), out4 (float32, n x 4), is_lepton (bool)) trimmed to the events."""
    n_max = int(n_max)
    chi, r, sb = (np.zeros(n_max) for _ in range(3))
    out4 = np.zeros((n_max, 4), dtype=np.float32)
    lep = np.zeros(n_max, dtype=np.uint8)
    n, fb = C.c_int64(0), C.c_ulonglong(0)
    _check(lib().qed_batch_mlp_last(batch, n_max, chi.ctypes.data, r.ctypes.data, sb.ctypes.data, out4.ctypes.data,
                                    lep.ctypes.data, C.byref(n), C.byref(fb)), "qed_batch_mlp_last")
    k = min(n_max, n.value)
    return n.value, fb.value, {"chi": chi[:k], "r": r[:k], "s_beta": sb[:k], "out4": out4[:k],
                               "is_lepton": lep[:k].astype(bool)}
