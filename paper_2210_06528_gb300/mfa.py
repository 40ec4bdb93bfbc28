"""Thin ctypes binding of the MFA C ABI (include/mfa.h).

Argument marshalling only: every step of the fit runs in the CUDA library.
Loading fails loudly when the library has not been built; there is no CPU
path.  PyTorch supplies device memory (tensor data pointers) and streams.

Function names match the C entry points; ``Handle`` and ``Model`` wrap them.
Grid arrays use the library's layout: shape (M_{d-1}, ..., M_0), C order.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

MFA_OK = 0
MFA_NOT_CONVERGED = 1
MFA_ERR_ARG = -1
MFA_ERR_LAYOUT = -2
MFA_ERR_OOM = -3
MFA_ERR_CUDA = -4
MFA_ERR_NOT_SPD = -5
MFA_ERR_DIVERGED = -6
MFA_ERR_NONFINITE = -7
MFA_ERR_UNSUPPORTED = -8
MFA_ERR_TIMEOUT = -9
MFA_ERR_IO = -10
MFA_SAVE_STATE = 1
MFA_F32, MFA_F64 = 0, 1
MFA_PREC_FP64, MFA_PREC_MIXED, MFA_PREC_FP32 = 0, 1, 2
MFA_KNOTS_FLOATING, MFA_KNOTS_CLAMPED = 0, 1
MFA_MAX_DEGREE = 7
MFA_UPDATE_AVERAGE, MFA_UPDATE_OWNER = 0, 1

MFA_TRACE_CLASSES = 16


class mfa_layout(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("degree", ctypes.c_int32), ("npts", ctypes.c_int64 * 3),
                ("nspans", ctypes.c_int32 * 3), ("nsub", ctypes.c_int32 * 3),
                ("core_spans", ctypes.POINTER(ctypes.c_int32) * 3), ("overlap", ctypes.c_int32 * 3),
                ("precision", ctypes.c_int32), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("knots", ctypes.c_int32), ("weights", ctypes.POINTER(ctypes.c_double) * 3)]


class mfa_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("dP_rel", ctypes.c_double),
                ("jump_max", ctypes.c_double), ("rms_decoded", ctypes.c_double),
                ("maxabs_decoded", ctypes.c_double), ("data_range", ctypes.c_double),
                ("jump_orders", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("jump_deriv", ctypes.c_double * (MFA_MAX_DEGREE + 1))]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("pad_", "jump_deriv")}
        d["jump_deriv"] = [self.jump_deriv[r] for r in range(self.jump_orders)]
        return d


class mfa_instance(ctypes.Structure):
    """One independent fit of a batch (see mfa_encode_batch)."""
    _fields_ = [("dim", ctypes.c_int32), ("degree", ctypes.c_int32), ("npts", ctypes.c_int64 * 3),
                ("nspans", ctypes.c_int32 * 3), ("q_offset", ctypes.c_int64)]


class mfa_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mfa_server_stats_t(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_int64), ("reserved", ctypes.c_int64), ("peak_reserved", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("resident_models", ctypes.c_int64), ("encode_jobs", ctypes.c_int64),
                ("decode_jobs", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MFAError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the built library (``__graft_entry__.build()`` or
    ``python -m paper_2210_06528_gb300.build`` makes it)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"MFA CUDA library not built: {path} is missing (run the build first)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.mfa_create.argtypes = [ctypes.c_int, P, ctypes.POINTER(P)]
    lib.mfa_destroy.argtypes = [P]
    lib.mfa_encode.argtypes = [P, ctypes.POINTER(mfa_layout), P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)]
    lib.mfa_schwarz_iterate.argtypes = [P, P, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                        ctypes.POINTER(mfa_report)]
    lib.mfa_interface_jumps.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(mfa_report)]
    lib.mfa_interface_jumps.restype = ctypes.c_int
    lib.mfa_decode.argtypes = [P, P, P, ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int]
    lib.mfa_encode_plain.argtypes = [P, ctypes.POINTER(mfa_layout), P, ctypes.c_int, ctypes.c_int, ctypes.c_int32,
                                     ctypes.c_double, ctypes.POINTER(mfa_report), ctypes.POINTER(P)]
    lib.mfa_residual.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(mfa_report)]
    lib.mfa_get_ctrl.argtypes = [P, P, P, ctypes.c_int64]
    lib.mfa_get_ctrl_async.argtypes = [P, P, P, ctypes.c_int64]
    lib.mfa_num_ctrl.argtypes = [P]
    lib.mfa_num_ctrl.restype = ctypes.c_int64
    lib.mfa_free.argtypes = [P]
    lib.mfa_sync.argtypes = [P]
    lib.mfa_status_string.argtypes = [ctypes.c_int]
    lib.mfa_status_string.restype = ctypes.c_char_p
    lib.mfa_axis_layout.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    lib.mfa_axis_layout.restype = ctypes.c_int
    lib.mfa_decode_grid_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int32), P, P, P]
    lib.mfa_decode_grid_noalloc.restype = ctypes.c_int
    lib.mfa_trace_enable.argtypes = [P, ctypes.c_int]
    lib.mfa_trace_enable.restype = ctypes.c_int
    lib.mfa_trace_read.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    lib.mfa_trace_read.restype = ctypes.c_int
    lib.mfa_trace_name.argtypes = [ctypes.c_int32]
    lib.mfa_trace_name.restype = ctypes.c_char_p
    lib.mfa_encode_batch.argtypes = [P, ctypes.c_int32, ctypes.POINTER(mfa_instance), P, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(P)]
    lib.mfa_batch_refit.argtypes = [P, P, P, ctypes.c_int]
    lib.mfa_batch_num_ctrl.argtypes = [P]
    lib.mfa_batch_num_ctrl.restype = ctypes.c_int64
    lib.mfa_batch_ctrl_offsets.argtypes = [P, P]
    lib.mfa_batch_get_ctrl.argtypes = [P, P, P, ctypes.c_int64]
    lib.mfa_batch_residual.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, P]
    lib.mfa_batch_decode.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int]
    lib.mfa_batch_free.argtypes = [P]
    lib.mfa_set_update_rule.argtypes = [P, P, ctypes.c_int]
    lib.mfa_save.argtypes = [P, P, ctypes.c_char_p, ctypes.c_int]
    lib.mfa_save.restype = ctypes.c_int
    lib.mfa_load.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(P)]
    lib.mfa_load.restype = ctypes.c_int
    lib.mfa_batch_tile_sizes.argtypes = [P, P, P]
    lib.mfa_batch_tile_sizes.restype = ctypes.c_int
    lib.mfa_batch_info.argtypes = [P, P]
    lib.mfa_batch_info.restype = ctypes.c_int
    lib.mfa_gram_condition.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P]
    lib.mfa_gram_condition.restype = ctypes.c_int
    lib.mfa_batch_group_tuning.argtypes = [P, ctypes.c_int32, P]
    lib.mfa_batch_group_tuning.restype = ctypes.c_int
    lib.mfa_batch_decode_points.argtypes = [P, P, ctypes.c_int32, P, P, P, P, ctypes.c_int]
    lib.mfa_server_create.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(P)]
    lib.mfa_server_encode.argtypes = [P, ctypes.POINTER(mfa_instance), P, ctypes.c_int]
    lib.mfa_server_encode.restype = ctypes.c_int64
    lib.mfa_server_decode.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, P]
    lib.mfa_server_decode.restype = ctypes.c_int64
    lib.mfa_server_wait.argtypes = [P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(mfa_request_info)]
    lib.mfa_server_release.argtypes = [P, ctypes.c_int64]
    lib.mfa_server_num_ctrl.argtypes = [P, ctypes.c_int64]
    lib.mfa_server_num_ctrl.restype = ctypes.c_int64
    lib.mfa_server_get_ctrl.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64]
    lib.mfa_server_stats.argtypes = [P, ctypes.POINTER(mfa_server_stats_t)]
    lib.mfa_server_destroy.argtypes = [P]
    for name in ["mfa_create", "mfa_destroy", "mfa_encode", "mfa_schwarz_iterate", "mfa_decode", "mfa_residual",
                 "mfa_get_ctrl", "mfa_get_ctrl_async", "mfa_free", "mfa_sync", "mfa_encode_plain", "mfa_encode_batch", "mfa_batch_refit",
                 "mfa_batch_ctrl_offsets", "mfa_batch_get_ctrl", "mfa_batch_residual", "mfa_batch_decode",
                 "mfa_batch_free", "mfa_batch_decode_points", "mfa_set_update_rule", "mfa_server_create", "mfa_server_wait",
                 "mfa_server_release", "mfa_server_get_ctrl", "mfa_server_stats", "mfa_server_destroy"]:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().mfa_status_string(int(code)).decode()


def _check(rc: int, where: str, ok=(MFA_OK,)) -> int:
    if rc not in ok:
        raise MFAError(rc, where)
    return rc


# ---------------------------------------------------------------------------
# C-named wrappers (argument marshalling only)
# ---------------------------------------------------------------------------

def ncp_of(degree, nspans, nsub, knots=MFA_KNOTS_FLOATING):
    """Control points of one axis: nspans + degree, plus (degree - 1) per
    interface with clamped interface knots."""
    n = int(nspans) + int(degree)
    if knots == MFA_KNOTS_CLAMPED and degree > 1:
        n += (int(degree) - 1) * (int(nsub) - 1)
    return n


def make_layout(dim, degree, npts, nspans, nsub, overlap, precision=MFA_PREC_FP64, core_spans=None, lo=None,
                hi=None, knots=MFA_KNOTS_FLOATING, weights=None):
    """Build an mfa_layout; the returned object keeps the core and weight
    arrays alive.  weights: None or one array of n_a positive weights per axis
    (separable NURBS weights)."""
    lay = mfa_layout()
    lay.dim = dim
    lay.degree = degree
    lay.knots = int(knots)
    keep = []
    for a in range(3):
        lay.npts[a] = int(npts[a]) if a < dim else 1
        lay.nspans[a] = int(nspans[a]) if a < dim else 1
        lay.nsub[a] = int(nsub[a]) if a < dim else 1
        lay.overlap[a] = int(overlap[a] if not np.isscalar(overlap) else overlap) if a < dim else 0
        lay.lo[a] = float(lo[a]) if lo is not None and a < dim else 0.0
        lay.hi[a] = float(hi[a]) if hi is not None and a < dim else 1.0
        if core_spans is not None and a < dim and core_spans[a] is not None:
            arr = (ctypes.c_int32 * len(core_spans[a]))(*[int(c) for c in core_spans[a]])
            keep.append(arr)
            lay.core_spans[a] = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32))
        else:
            lay.core_spans[a] = ctypes.POINTER(ctypes.c_int32)()
        if weights is not None and a < dim and weights[a] is not None:
            warr = np.ascontiguousarray(weights[a], dtype=np.float64)
            keep.append(warr)
            lay.weights[a] = warr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        else:
            lay.weights[a] = ctypes.POINTER(ctypes.c_double)()
    lay.precision = precision
    lay._keep = keep
    return lay


def mfa_axis_layout(npts: int, nspans: int, degree: int, nsub: int, overlap: int, core_spans=None,
                    knots: int = MFA_KNOTS_FLOATING):
    """Host-built layout of one axis (no device needed): returns (rows, owner)
    with rows[s] = (a, b, w0, w1, k0, k1, l0, nL, oU, nU) per subdomain and
    owner[g] the Greville owner of control point g; raises MFAError on a
    rejection."""
    rows = (ctypes.c_int32 * (10 * max(nsub, 1)))()
    n = ncp_of(degree, nspans, nsub, knots)
    owner = (ctypes.c_int32 * max(n, 1))()
    cores = None
    if core_spans is not None:
        cores = (ctypes.c_int32 * len(core_spans))(*[int(c) for c in core_spans])
    _check(load().mfa_axis_layout(int(npts), int(nspans), int(degree), int(nsub), cores, int(overlap), int(knots),
                                  rows, int(nsub), owner), "mfa_axis_layout")
    return np.array(rows, dtype=np.int64).reshape(nsub, 10), np.array(owner, dtype=np.int64)


def mfa_create(device: int = 0, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().mfa_create(device, ctypes.c_void_p(stream), ctypes.byref(h)), "mfa_create")
    return h.value


def mfa_destroy(h: int) -> None:
    _check(load().mfa_destroy(ctypes.c_void_p(h)), "mfa_destroy")


def mfa_encode(h: int, layout: mfa_layout, q_ptr: int, q_dtype: int, q_on_device: bool) -> int:
    m = ctypes.c_void_p()
    _check(load().mfa_encode(ctypes.c_void_p(h), ctypes.byref(layout), ctypes.c_void_p(q_ptr), q_dtype,
                             int(q_on_device), ctypes.byref(m)), "mfa_encode")
    return m.value


def mfa_schwarz_iterate(h: int, m: int, max_iters: int, tol_dP: float, tol_rms_stall: float = 0.0):
    rep = mfa_report()
    rc = load().mfa_schwarz_iterate(ctypes.c_void_p(h), ctypes.c_void_p(m), int(max_iters), float(tol_dP),
                                    float(tol_rms_stall), ctypes.byref(rep))
    _check(rc, "mfa_schwarz_iterate", ok=(MFA_OK, MFA_NOT_CONVERGED))
    return rc, rep


def mfa_interface_jumps(h: int, m: int, max_order: int) -> mfa_report:
    rep = mfa_report()
    _check(load().mfa_interface_jumps(ctypes.c_void_p(h), ctypes.c_void_p(m), int(max_order), ctypes.byref(rep)),
           "mfa_interface_jumps")
    return rep


def mfa_encode_plain(h: int, layout: mfa_layout, q_ptr: int, q_dtype: int, q_on_device: bool, max_iters: int,
                     tol_dP: float):
    """Per-subdomain comparator form (FP64); returns (model, rc, report)."""
    m = ctypes.c_void_p()
    rep = mfa_report()
    rc = load().mfa_encode_plain(ctypes.c_void_p(h), ctypes.byref(layout), ctypes.c_void_p(q_ptr), q_dtype,
                                 int(q_on_device), int(max_iters), float(tol_dP), ctypes.byref(rep), ctypes.byref(m))
    _check(rc, "mfa_encode_plain", ok=(MFA_OK, MFA_NOT_CONVERGED))
    return m.value, rc, rep


def make_instances(specs) -> "ctypes.Array":
    """specs: iterable of dicts with dim, degree, npts, nspans, q_offset."""
    specs = list(specs)
    arr = (mfa_instance * len(specs))()
    for k, sp in enumerate(specs):
        d = int(sp["dim"])
        arr[k].dim = d
        arr[k].degree = int(sp["degree"])
        npts = list(sp["npts"]) + [1] * (3 - d)
        nsp = list(sp["nspans"]) + [1] * (3 - d)
        for a in range(3):
            arr[k].npts[a] = int(npts[a])
            arr[k].nspans[a] = int(nsp[a])
        arr[k].q_offset = int(sp["q_offset"])
    return arr


def mfa_encode_batch(h: int, inst, q_ptr: int, q_dtype: int, q_on_device: bool, precision: int) -> int:
    b = ctypes.c_void_p()
    _check(load().mfa_encode_batch(ctypes.c_void_p(h), len(inst), inst, ctypes.c_void_p(q_ptr), q_dtype,
                                   int(q_on_device), int(precision), ctypes.byref(b)), "mfa_encode_batch")
    return b.value


def mfa_batch_refit(h: int, b: int, q_ptr: int, q_dtype: int) -> None:
    _check(load().mfa_batch_refit(ctypes.c_void_p(h), ctypes.c_void_p(b), ctypes.c_void_p(q_ptr), q_dtype),
           "mfa_batch_refit")


def mfa_batch_num_ctrl(b: int) -> int:
    return int(load().mfa_batch_num_ctrl(ctypes.c_void_p(b)))


def mfa_batch_ctrl_offsets(b: int, count: int) -> np.ndarray:
    off = np.empty(count + 1, dtype=np.int64)
    _check(load().mfa_batch_ctrl_offsets(ctypes.c_void_p(b), off.ctypes.data), "mfa_batch_ctrl_offsets")
    return off


def mfa_batch_get_ctrl(h: int, b: int) -> np.ndarray:
    n = mfa_batch_num_ctrl(b)
    out = np.empty(n, dtype=np.float64)
    _check(load().mfa_batch_get_ctrl(ctypes.c_void_p(h), ctypes.c_void_p(b), out.ctypes.data, n),
           "mfa_batch_get_ctrl")
    return out


def mfa_batch_residual(h: int, b: int, count: int, q_ptr: int, q_dtype: int, q_on_device: bool):
    rms = np.empty(count, dtype=np.float64)
    mx = np.empty(count, dtype=np.float64)
    _check(load().mfa_batch_residual(ctypes.c_void_p(h), ctypes.c_void_p(b), ctypes.c_void_p(q_ptr), q_dtype,
                                     int(q_on_device), rms.ctypes.data, mx.ctypes.data), "mfa_batch_residual")
    return rms, mx


def mfa_batch_decode(h: int, b: int, out_ptr: int, out_dtype: int, out_on_device: bool) -> None:
    _check(load().mfa_batch_decode(ctypes.c_void_p(h), ctypes.c_void_p(b), ctypes.c_void_p(out_ptr), out_dtype,
                                   int(out_on_device)), "mfa_batch_decode")


def mfa_set_update_rule(h: int, m: int, rule: int) -> None:
    _check(load().mfa_set_update_rule(ctypes.c_void_p(h), ctypes.c_void_p(m), int(rule)), "mfa_set_update_rule")


def mfa_save(h: int, m: int, path: str, flags: int = 0) -> None:
    _check(load().mfa_save(ctypes.c_void_p(h), ctypes.c_void_p(m), os.fsencode(path), int(flags)), "mfa_save")


def mfa_load(h: int, path: str) -> int:
    m = ctypes.c_void_p()
    _check(load().mfa_load(ctypes.c_void_p(h), os.fsencode(path), ctypes.byref(m)), "mfa_load")
    return m.value


def saved_layout(path: str) -> mfa_layout:
    """The layout stored in a saved model's header (dimension, degree, grid,
    spans, subdomains, overlap, precision, box, knots at the interfaces and
    NURBS weights)."""
    import struct
    with open(path, "rb") as f:
        head = f.read(192)
        fields = struct.unpack("<8s8i3q12i6d2d2q", head)
        version, dim, degree, prec = fields[1], fields[2], fields[3], fields[4]
        knots = fields[8] if version >= 2 else MFA_KNOTS_FLOATING
        npts = fields[9:12]
        nspans, nsub, overlap = fields[12:15], fields[15:18], fields[18:21]
        wmask = fields[21] if version >= 2 else 0
        lo, hi = fields[22:25], fields[25:28]
        cores = [list(struct.unpack(f"<{nsub[a]}i", f.read(4 * nsub[a]))) for a in range(dim)]
        weights = None
        if wmask:
            weights = []
            for a in range(dim):
                if wmask & (1 << a):
                    n = ncp_of(degree, nspans[a], nsub[a], knots)
                    weights.append(np.frombuffer(f.read(8 * n), dtype="<f8").copy())
                else:
                    weights.append(None)
    return make_layout(dim, degree, list(npts[:dim]), list(nspans[:dim]), list(nsub[:dim]), list(overlap[:dim]), prec,
                       core_spans=cores, lo=list(lo[:dim]), hi=list(hi[:dim]), knots=knots, weights=weights)


class MfaBatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("groups", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("refined", ctypes.c_int32), ("items", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("points", ctypes.c_int64), ("ctrl", ctypes.c_int64)]


def mfa_gram_condition(npts: int, nspans: int, degree: int) -> float:
    """Host estimate of one axis's cond(N^T N) (the FP32 refinement rule's input)."""
    out = ctypes.c_double()
    _check(load().mfa_gram_condition(ctypes.c_int64(npts), ctypes.c_int32(nspans), ctypes.c_int32(degree),
                                     ctypes.byref(out)), "mfa_gram_condition")
    return out.value


def mfa_batch_info(b: int) -> dict:
    info = MfaBatchInfo()
    _check(load().mfa_batch_info(ctypes.c_void_p(b), ctypes.byref(info)), "mfa_batch_info")
    return {f: getattr(info, f) for f, _ in MfaBatchInfo._fields_ if f != "reserved"}


MFA_TUNE_CANDIDATES = 10


class MfaGroupTuning(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("degree", ctypes.c_int32), ("instances", ctypes.c_int32),
                ("tile_c", ctypes.c_int32), ("tile_s", ctypes.c_int32), ("tile_e", ctypes.c_int32),
                ("fused", ctypes.c_int32), ("item_pts", ctypes.c_int32), ("chosen_ms", ctypes.c_float),
                ("candidate_ms", ctypes.c_float * MFA_TUNE_CANDIDATES)]


def mfa_batch_group_tuning(b: int, group: int):
    """(rc, dict) of one group's autotuned choice and its timed candidates."""
    t = MfaGroupTuning()
    rc = load().mfa_batch_group_tuning(ctypes.c_void_p(b), int(group), ctypes.byref(t))
    _check(rc, "mfa_batch_group_tuning", ok=(MFA_OK, MFA_NOT_CONVERGED))
    out = {f: getattr(t, f) for f, _ in MfaGroupTuning._fields_ if f != "candidate_ms"}
    out["candidate_ms"] = [float(x) for x in t.candidate_ms]
    return rc, out


def mfa_batch_tile_sizes(b: int):
    """(rc, [projection, solve, decode] block sizes, 3x3 candidate fit times in ms)."""
    sizes = (ctypes.c_int32 * 3)()
    ms = (ctypes.c_float * 9)()
    rc = load().mfa_batch_tile_sizes(ctypes.c_void_p(b), sizes, ms)
    return rc, list(sizes), np.array(list(ms)).reshape(3, 3)


def mfa_batch_decode_points(h: int, b: int, qinst, pt_off, pts, out) -> None:
    """Host arrays: qinst int32 [nq], pt_off int64 [nq + 1], pts float64 [npts, 3], out float64 [npts];
    or all four as contiguous CUDA tensors of those types."""
    if hasattr(pts, "is_cuda") and pts.is_cuda:
        for t, dt in ((qinst, "torch.int32"), (pt_off, "torch.int64"), (pts, "torch.float64"), (out, "torch.float64")):
            if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous() and str(t.dtype) == dt):
                raise TypeError("device decode: qinst int32, pt_off int64, pts and out float64, contiguous CUDA")
        _check(load().mfa_batch_decode_points(ctypes.c_void_p(h), ctypes.c_void_p(b), int(qinst.numel()),
                                              ctypes.c_void_p(qinst.data_ptr()), ctypes.c_void_p(pt_off.data_ptr()),
                                              ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1),
               "mfa_batch_decode_points")
        return
    qinst = np.ascontiguousarray(qinst, dtype=np.int32)
    pt_off = np.ascontiguousarray(pt_off, dtype=np.int64)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise TypeError("out must be a contiguous float64 array")
    _check(load().mfa_batch_decode_points(ctypes.c_void_p(h), ctypes.c_void_p(b), len(qinst), qinst.ctypes.data,
                                          pt_off.ctypes.data, pts.ctypes.data, out.ctypes.data, 0),
           "mfa_batch_decode_points")


def mfa_server_create(device: int, workers: int, mem_budget: int, max_batch: int) -> int:
    s = ctypes.c_void_p()
    _check(load().mfa_server_create(int(device), int(workers), int(mem_budget), int(max_batch), ctypes.byref(s)),
           "mfa_server_create")
    return s.value


def mfa_server_encode(s: int, inst, q_ptr: int, precision: int) -> int:
    rid = load().mfa_server_encode(ctypes.c_void_p(s), ctypes.byref(inst), ctypes.c_void_p(q_ptr), int(precision))
    if rid < 0:
        raise MFAError(int(rid), "mfa_server_encode")
    return int(rid)


def mfa_server_decode(s: int, model: int, npts: int, pts_ptr: int, out_ptr: int) -> int:
    rid = load().mfa_server_decode(ctypes.c_void_p(s), int(model), int(npts), ctypes.c_void_p(pts_ptr),
                                   ctypes.c_void_p(out_ptr))
    if rid < 0:
        raise MFAError(int(rid), "mfa_server_decode")
    return int(rid)


def mfa_server_wait(s: int, rid: int, timeout_s: float = 0.0):
    info = mfa_request_info()
    rc = load().mfa_server_wait(ctypes.c_void_p(s), int(rid), float(timeout_s), ctypes.byref(info))
    return rc, info


def mfa_server_release(s: int, model: int) -> None:
    _check(load().mfa_server_release(ctypes.c_void_p(s), int(model)), "mfa_server_release")


def mfa_server_num_ctrl(s: int, model: int) -> int:
    return int(load().mfa_server_num_ctrl(ctypes.c_void_p(s), int(model)))


def mfa_server_get_ctrl(s: int, model: int) -> np.ndarray:
    n = mfa_server_num_ctrl(s, model)
    if n < 0:
        raise MFAError(n, "mfa_server_num_ctrl")
    out = np.empty(n, dtype=np.float64)
    _check(load().mfa_server_get_ctrl(ctypes.c_void_p(s), int(model), out.ctypes.data, n), "mfa_server_get_ctrl")
    return out


def mfa_server_stats(s: int) -> dict:
    st = mfa_server_stats_t()
    _check(load().mfa_server_stats(ctypes.c_void_p(s), ctypes.byref(st)), "mfa_server_stats")
    return st.as_dict()


def mfa_server_destroy(s: int) -> None:
    _check(load().mfa_server_destroy(ctypes.c_void_p(s)), "mfa_server_destroy")


def mfa_batch_free(b: int) -> None:
    _check(load().mfa_batch_free(ctypes.c_void_p(b)), "mfa_batch_free")


def mfa_decode(h: int, m: int, pts_ptr: int, npts_q: int, deriv, out_ptr: int, out_dtype: int,
               out_on_device: bool) -> None:
    d = None
    if deriv is not None:
        d = (ctypes.c_int32 * 3)(*(list(deriv) + [0] * (3 - len(deriv))))
    _check(load().mfa_decode(ctypes.c_void_p(h), ctypes.c_void_p(m), ctypes.c_void_p(pts_ptr), int(npts_q),
                             ctypes.cast(d, ctypes.c_void_p) if d is not None else None, ctypes.c_void_p(out_ptr),
                             out_dtype, int(out_on_device)), "mfa_decode")


def mfa_residual(h: int, m: int, q_ptr: int, q_dtype: int, q_on_device: bool) -> mfa_report:
    rep = mfa_report()
    _check(load().mfa_residual(ctypes.c_void_p(h), ctypes.c_void_p(m), ctypes.c_void_p(q_ptr), q_dtype,
                               int(q_on_device), ctypes.byref(rep)), "mfa_residual")
    return rep


def mfa_num_ctrl(m: int) -> int:
    return int(load().mfa_num_ctrl(ctypes.c_void_p(m)))


def mfa_get_ctrl(h: int, m: int, out=None):
    """Control points as FP64 into ``out`` (a host numpy array or CPU torch
    tensor of at least mfa_num_ctrl values, e.g. pinned), or a new array."""
    n = mfa_num_ctrl(m)
    if out is None:
        out = np.empty(n, dtype=np.float64)
    ptr, code, dev, keep = _ptr_dtype(out)
    if dev or code != MFA_F64 or keep is not out:
        raise TypeError("control points are read into a contiguous host float64 buffer")
    cap = out.numel() if hasattr(out, "numel") else out.size
    _check(load().mfa_get_ctrl(ctypes.c_void_p(h), ctypes.c_void_p(m), ptr, cap), "mfa_get_ctrl")
    return out


def mfa_get_ctrl_async(h: int, m: int, out):
    """Enqueue the read of the control points into ``out`` (a host float64
    buffer, pinned for an asynchronous copy); the values are there once
    mfa_sync(h) has returned."""
    ptr, code, dev, keep = _ptr_dtype(out)
    if dev or code != MFA_F64 or keep is not out:
        raise TypeError("control points are read into a contiguous host float64 buffer")
    cap = out.numel() if hasattr(out, "numel") else out.size
    _check(load().mfa_get_ctrl_async(ctypes.c_void_p(h), ctypes.c_void_p(m), ptr, cap), "mfa_get_ctrl_async")
    return out


def mfa_free(m: int) -> None:
    _check(load().mfa_free(ctypes.c_void_p(m)), "mfa_free")


def mfa_sync(h: int) -> int:
    return load().mfa_sync(ctypes.c_void_p(h))


def mfa_decode_grid_noalloc(dim: int, degree: int, npts, nspans, ctrl_ptr: int, out_ptr: int, stream: int = 0) -> None:
    """Grid decode into caller-owned device buffers using only the library's
    fixed static scratch (no allocation); see include/mfa.h."""
    n = (ctypes.c_int64 * 3)(*[int(x) for x in npts] + [1] * (3 - len(npts)))
    s = (ctypes.c_int32 * 3)(*[int(x) for x in nspans] + [1] * (3 - len(nspans)))
    _check(load().mfa_decode_grid_noalloc(int(dim), int(degree), n, s, ctypes.c_void_p(ctrl_ptr),
                                          ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream)),
           "mfa_decode_grid_noalloc")


def mfa_trace_enable(h: int, enable: bool) -> None:
    _check(load().mfa_trace_enable(ctypes.c_void_p(h), int(enable)), "mfa_trace_enable")


def mfa_trace_read(h: int, cls: int):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().mfa_trace_read(ctypes.c_void_p(h), int(cls), ctypes.byref(ms), ctypes.byref(n)), "mfa_trace_read")
    return ms.value, n.value


def mfa_trace_name(cls: int) -> str:
    return load().mfa_trace_name(int(cls)).decode()


def trace_table(h: int) -> dict:
    """{class name: (total ms, launches)} for every kernel class."""
    out = {}
    for c in range(MFA_TRACE_CLASSES):
        ms, n = mfa_trace_read(h, c)
        if n:
            out[mfa_trace_name(c)] = (ms, n)
    return out


# ---------------------------------------------------------------------------
# convenience classes
# ---------------------------------------------------------------------------

def _ptr_dtype(q):
    """(pointer, dtype code, on_device, keepalive) for a torch tensor or numpy array."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(q, torch.Tensor):
        if not q.is_contiguous():
            q = q.contiguous()
        if q.dtype == torch.float32:
            code = MFA_F32
        elif q.dtype == torch.float64:
            code = MFA_F64
        else:
            raise TypeError("data must be float32 or float64")
        return q.data_ptr(), code, q.is_cuda, q
    a = np.ascontiguousarray(q)
    if a.dtype == np.float32:
        code = MFA_F32
    elif a.dtype == np.float64:
        code = MFA_F64
    else:
        raise TypeError("data must be float32 or float64")
    return a.ctypes.data, code, False, a


class Handle:
    """A library handle on one device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self.stream = stream
        self.h = mfa_create(device, stream)

    def encode(self, q, layout: mfa_layout) -> "Model":
        ptr, code, dev, keep = _ptr_dtype(q)
        m = mfa_encode(self.h, layout, ptr, code, dev)
        return Model(self, m, layout)

    def encode_batch(self, specs, q, precision: int = MFA_PREC_MIXED) -> "Batch":
        """Fit many independent grids at once (specs: dim, degree, npts, nspans, q_offset per instance)."""
        inst = make_instances(specs)
        ptr, code, dev, keep = _ptr_dtype(q)
        b = mfa_encode_batch(self.h, inst, ptr, code, dev, precision)
        return Batch(self, b, len(inst))

    def load(self, path: str) -> "Model":
        """A model saved with Model.save, rebuilt on this handle's device."""
        m = mfa_load(self.h, path)
        return Model(self, m, saved_layout(path))

    def encode_plain(self, q, layout: mfa_layout, max_iters: int, tol_dP: float):
        """Encode and iterate in the per-subdomain comparator form; returns (Model, rc, report)."""
        ptr, code, dev, keep = _ptr_dtype(q)
        m, rc, rep = mfa_encode_plain(self.h, layout, ptr, code, dev, max_iters, tol_dP)
        return Model(self, m, layout), rc, rep

    def sync(self) -> int:
        return mfa_sync(self.h)

    def close(self):
        if self.h:
            mfa_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Model:
    """A fitted MFA resident on the device."""

    def __init__(self, handle: Handle, m: int, layout: mfa_layout):
        self.handle = handle
        self.m = m
        self.dim = layout.dim
        self.degree = layout.degree
        self.npts = [int(layout.npts[a]) for a in range(self.dim)]
        self.ncp = [ncp_of(layout.degree, layout.nspans[a], layout.nsub[a], layout.knots) for a in range(self.dim)]

    def save(self, path: str, state: bool = False) -> None:
        """Write the model (and with state=True the Schwarz state, to iterate on after a load)."""
        mfa_save(self.handle.h, self.m, path, MFA_SAVE_STATE if state else 0)

    def set_update_rule(self, rule: int) -> None:
        """MFA_UPDATE_AVERAGE or MFA_UPDATE_OWNER; recomputes the current global control points."""
        mfa_set_update_rule(self.handle.h, self.m, rule)

    def iterate(self, max_iters: int, tol_dP: float = 0.0, tol_rms_stall: float = 0.0):
        """Schwarz iterations until dP_rel <= tol_dP or the decoded RMS stalls
        (|RMS_k - RMS_{k-1}| <= tol_rms_stall RMS_k); returns (rc, report)."""
        return mfa_schwarz_iterate(self.handle.h, self.m, max_iters, tol_dP, tol_rms_stall)

    def jumps(self, max_order: int) -> np.ndarray:
        """Largest interface jump of every derivative order 0..max_order (span units)."""
        rep = mfa_interface_jumps(self.handle.h, self.m, max_order)
        return np.array([rep.jump_deriv[r] for r in range(rep.jump_orders)])

    def ctrl(self, out=None):
        """Global control points (grid layout, reversed axes); with ``out`` a
        preallocated host float64 buffer is filled and returned as is."""
        if out is not None:
            return mfa_get_ctrl(self.handle.h, self.m, out)
        return mfa_get_ctrl(self.handle.h, self.m).reshape(tuple(reversed(self.ncp)))

    def ctrl_async(self, out):
        """Enqueue the read of the control points into the host float64
        buffer ``out``; it holds them once Handle.sync() has returned."""
        return mfa_get_ctrl_async(self.handle.h, self.m, out)

    def residual(self, q=None) -> mfa_report:
        """Decoded error statistics against ``q``; None uses the device copy
        encode() made of host data."""
        if q is None:
            return mfa_residual(self.handle.h, self.m, 0, MFA_F32, False)
        ptr, code, dev, keep = _ptr_dtype(q)
        return mfa_residual(self.handle.h, self.m, ptr, code, dev)

    def decode_grid(self, out):
        """Decode on the full data grid into ``out`` (torch tensor or numpy array)."""
        ptr, code, dev, keep = _ptr_dtype(out)
        mfa_decode(self.handle.h, self.m, 0, 0, None, ptr, code, dev)
        return out

    def decode_points(self, pts, out, deriv: Optional[Sequence[int]] = None):
        """Decode at scattered physical points pts[k, a] (host or device FP64)."""
        pptr, pcode, pdev, pkeep = _ptr_dtype(pts)
        if pcode != MFA_F64:
            raise TypeError("points must be float64")
        optr, ocode, odev, okeep = _ptr_dtype(out)
        n = pts.shape[0]
        mfa_decode(self.handle.h, self.m, pptr, n, deriv, optr, ocode, odev)
        return out

    def free(self):
        if self.m:
            mfa_free(self.m)
            self.m = None


class Batch:
    """A batch of independent fits (mfa_encode_batch); control points are
    concatenated in instance order."""

    def __init__(self, handle: Handle, b: int, count: int):
        self.handle = handle
        self.b = b
        self.count = count

    def offsets(self) -> np.ndarray:
        return mfa_batch_ctrl_offsets(self.b, self.count)

    def ctrl(self) -> np.ndarray:
        return mfa_batch_get_ctrl(self.handle.h, self.b)

    def refit(self, q) -> None:
        ptr, code, dev, keep = _ptr_dtype(q)
        if not dev:
            raise TypeError("refit takes device data")
        mfa_batch_refit(self.handle.h, self.b, ptr, code)

    def residual(self, q=None):
        if q is None:
            return mfa_batch_residual(self.handle.h, self.b, self.count, 0, MFA_F32, False)
        ptr, code, dev, keep = _ptr_dtype(q)
        return mfa_batch_residual(self.handle.h, self.b, self.count, ptr, code, dev)

    def decode(self, out):
        ptr, code, dev, keep = _ptr_dtype(out)
        mfa_batch_decode(self.handle.h, self.b, ptr, code, dev)
        return out

    def tile_sizes(self):
        return mfa_batch_tile_sizes(self.b)

    def info(self) -> dict:
        return mfa_batch_info(self.b)

    def group_tuning(self):
        """Autotuned choice of every (dimension, degree) group (after the first refit)."""
        return [mfa_batch_group_tuning(self.b, g)[1] for g in range(self.info()["groups"])]

    def decode_points(self, qinst, pt_off, pts, out=None):
        """Scattered decode: query k evaluates instance qinst[k] at pts[pt_off[k]:pt_off[k+1]]
        (parameters in [0,1], three per point); returns float64 values.  CUDA
        tensors (int32, int64, float64 [npts, 3], float64 out) stay on the device."""
        if hasattr(pts, "is_cuda") and pts.is_cuda:
            mfa_batch_decode_points(self.handle.h, self.b, qinst, pt_off, pts, out)
            return out
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        if out is None:
            out = np.empty(len(pts), dtype=np.float64)
        mfa_batch_decode_points(self.handle.h, self.b, qinst, pt_off, pts, out)
        return out

    def free(self):
        if self.b:
            mfa_batch_free(self.b)
            self.b = None


class Server:
    """Continuous-batching server (mfa_server_*): encode requests and decode
    queries from any thread; ids name requests and, for encodes, models.
    Buffers passed in must stay alive until the request is done; the object
    keeps references to them until wait() returns."""

    def __init__(self, device: int = 0, workers: int = 3, mem_budget: int = 8 << 30, max_batch: int = 64):
        self.s = mfa_server_create(device, workers, mem_budget, max_batch)
        self._keep = {}

    def encode(self, spec, q, precision: int = MFA_PREC_MIXED) -> int:
        inst = make_instances([dict(spec, q_offset=0)])[0]
        a = q if hasattr(q, "data_ptr") else np.ascontiguousarray(q, dtype=np.float32)
        ptr = a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        rid = mfa_server_encode(self.s, inst, ptr, precision)
        self._keep[rid] = a
        return rid

    def decode(self, model: int, pts, out) -> int:
        p = pts if hasattr(pts, "data_ptr") else np.ascontiguousarray(pts, dtype=np.float64)
        pp = p.data_ptr() if hasattr(p, "data_ptr") else p.ctypes.data
        op = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        n = (p.numel() if hasattr(p, "numel") else p.size) // 3
        rid = mfa_server_decode(self.s, model, n, pp, op)
        self._keep[rid] = (p, out)
        return rid

    def wait(self, rid: int, timeout_s: float = 0.0):
        rc, info = mfa_server_wait(self.s, rid, timeout_s)
        if rc != MFA_ERR_TIMEOUT:
            self._keep.pop(rid, None)
        return rc, info.as_dict()

    def release(self, model: int) -> None:
        mfa_server_release(self.s, model)

    def ctrl(self, model: int) -> np.ndarray:
        return mfa_server_get_ctrl(self.s, model)

    def stats(self) -> dict:
        return mfa_server_stats(self.s)

    def close(self):
        if self.s:
            mfa_server_destroy(self.s)
            self.s = None
            self._keep.clear()

