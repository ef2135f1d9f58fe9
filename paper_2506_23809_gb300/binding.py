"""Thin ctypes binding of libqc_eloc (include/qc_eloc.h), same names as the C ABI.

Argument marshalling only: tensors are passed as device pointers, the stream as
``torch.cuda.current_stream().cuda_stream``; every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing, loading
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqc_eloc.so")
LIB_CHECKED_PATH = os.path.join(HERE, "libqc_eloc_checked.so")

QC_OK, QC_PENDING = 0, 1
QC_FP64, QC_FP32_COMP = 0, 1
QC_SAMPLE, QC_FULL = 0, 1
QC_OPT_TIMING, QC_OPT_KERNEL, QC_OPT_FILTER_LOG2W, QC_OPT_WARPS, QC_OPT_UNROLL, QC_OPT_GRID = 1, 2, 3, 4, 5, 6
QC_OPT_PREFILTER = 7
QC_OPT_LEAN = 8
QC_OPT_CHUNK_PAIRS = 9
QC_OPT_JOIN = 10
QC_OPT_SCAN_COST = 11
QC_OPT_BETA_COST = 15
QC_OPT_COUNT_WORK = 12
QC_OPT_WAIT_LIMIT = 13
QC_OPT_ALPHA_SLOTS = 14
WORK_FIELDS = ("samples", "scan_rows", "tests", "probes", "hits_single", "hits_same", "hits_ab", "ctas",
               "hits_scanned", "beta_looked", "beta_groups")
QC_SRV_OPT_QUANTUM = 1
QC_SRV_OPT_OLDEST_PCT = 2
QC_SRV_OPT_WAVE_ROWS = 3
STATUS_NAMES = {0: "QC_OK", 1: "QC_PENDING", -1: "QC_ERR_ARG", -2: "QC_ERR_UNSORTED", -3: "QC_ERR_DUP",
                -4: "QC_ERR_NELEC", -5: "QC_ERR_OOM", -6: "QC_ERR_BUDGET", -7: "QC_ERR_CUDA",
                -8: "QC_ERR_ZERO_PSI", -9: "QC_ERR_MISSING", -10: "QC_ERR_TIMEOUT",
                -11: "QC_ERR_CAPACITY", -12: "QC_ERR_COUNTS", -13: "QC_ERR_BOUNDS"}


class QcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class qc_eloc_summary(ctypes.Structure):
    _fields_ = [("e_re", ctypes.c_double), ("e_im", ctypes.c_double), ("var", ctypes.c_double),
                ("w", ctypes.c_double), ("sum_ce_re", ctypes.c_double), ("sum_ce_im", ctypes.c_double),
                ("n_used", ctypes.c_uint64), ("n_pairs", ctypes.c_uint64), ("n_hits", ctypes.c_uint64),
                ("n_missing", ctypes.c_uint64), ("n_bad", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("status", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["energy"] = complex(self.e_re, self.e_im)
        return d


class qc_eloc_out(ctypes.Structure):
    _fields_ = [("eloc", ctypes.c_void_p), ("summary", ctypes.c_void_p), ("hit_count", ctypes.c_void_p),
                ("hit_rowsum", ctypes.c_void_p), ("hit_signsum", ctypes.c_void_p),
                ("hit_cursor", ctypes.c_void_p), ("hit_list", ctypes.c_void_p), ("hit_list_cap", ctypes.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libqc_eloc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libqc_eloc.so not found at {path}: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.qc_eloc_create.argtypes = [P, P, f64, i32, i32, i32, i32, ctypes.POINTER(P)]
    lib.qc_eloc_create.restype = i32
    lib.qc_eloc_destroy.argtypes = [P]
    lib.qc_eloc_destroy.restype = i32
    lib.qc_eloc_last_error.argtypes = [P]
    lib.qc_eloc_last_error.restype = ctypes.c_char_p
    lib.qc_eloc_reserve.argtypes = [P, i64, i64]
    lib.qc_eloc_reserve.restype = i32
    lib.qc_eloc_set_option.argtypes = [P, i32, i64]
    lib.qc_eloc_set_option.restype = i32
    lib.qc_eloc_pairs_per_sample.argtypes = [P]
    lib.qc_eloc_pairs_per_sample.restype = i64
    lib.qc_eloc_eval.argtypes = [P, P, P, P, i64, P, P, i64, ctypes.POINTER(qc_eloc_out), P]
    lib.qc_eloc_eval.restype = i32
    lib.qc_eloc_timings.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.qc_eloc_timings.restype = i32
    lib.qc_eloc_last_config.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.qc_eloc_last_config.restype = i32
    lib.qc_eloc_work.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), i32]
    lib.qc_eloc_work.restype = i32
    lib.qc_test_fail_alloc.argtypes = [i64]
    lib.qc_test_fail_alloc.restype = i32
    lib.qc_eloc_eval_static.argtypes = [P, P, f64, i32, i32, P, P, P, i64, P, P, P]
    lib.qc_eloc_eval_static.restype = i32
    lib.qc_eloc_grad.argtypes = [P, P, P, i64, P, i64, P, P, P]
    lib.qc_eloc_grad.restype = i32
    lib.qc_eloc_export.argtypes = [P, P, i64, P, P, P, P]
    lib.qc_eloc_export.restype = i32
    lib.qc_eloc_apply.argtypes = [P, P, P, i64, P, P, P, P, P, P]
    lib.qc_eloc_apply.restype = i32
    lib.qc_probe_peaks.argtypes = [P, P, P]
    lib.qc_probe_peaks.restype = i32
    lib.qc_dedup_workspace_bytes.argtypes = [i64]
    lib.qc_dedup_workspace_bytes.restype = i64
    lib.qc_dedup.argtypes = [P, i64, i32, P, P, P, P, ctypes.c_size_t, P]
    lib.qc_dedup.restype = i32
    lib.qc_batch_create.argtypes = [P, i32, ctypes.POINTER(P)]
    lib.qc_batch_destroy.argtypes = [P]
    lib.qc_batch_last_error.argtypes = [P]
    lib.qc_batch_last_error.restype = ctypes.c_char_p
    lib.qc_batch_set_inputs.argtypes = [P, i32, P, P, P, i64, P]
    lib.qc_batch_set_config.argtypes = [P, i32, i32, i32]
    lib.qc_batch_config.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.qc_batch_eval.argtypes = [P, P, P]
    lib.qc_batch_graph_launch.argtypes = [P, P, P]
    lib.qc_batch_timings.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.qc_batch_autotune.argtypes = [P, P, i32, ctypes.POINTER(ctypes.c_int64)]
    lib.qc_batch_set_chunk_pairs.argtypes = [P, i64]
    lib.qc_batch_set_rows.argtypes = [P, i32, i64, i64]
    for f in ("qc_batch_create", "qc_batch_destroy", "qc_batch_set_inputs", "qc_batch_set_config",
              "qc_batch_config", "qc_batch_eval", "qc_batch_graph_launch", "qc_batch_timings", "qc_batch_autotune",
              "qc_batch_set_chunk_pairs", "qc_batch_set_rows"):
        getattr(lib, f).restype = i32
    _lib = lib
    return lib


def _check(st, handle=None):
    if st != QC_OK:
        lib = load_library()
        msg = lib.qc_eloc_last_error(handle).decode() if lib else ""
        raise QcError(st, msg)


@dataclass
class QcHandle:
    """A qc_eloc* plus a page-locked summary buffer reused by every evaluation."""
    ptr: ctypes.c_void_p
    n_orb: int
    n_elec: int
    precision: int
    mode: int
    summary_buf: object  # torch pinned uint8 tensor

    def summary_struct(self) -> qc_eloc_summary:
        return qc_eloc_summary.from_address(self.summary_buf.data_ptr())


def qc_eloc_create(h, eri, e_core: float, n_orb: int, n_elec: int, precision: int = QC_FP64,
                   mode: int = QC_SAMPLE) -> QcHandle:
    import torch
    lib = load_library()
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    out = ctypes.c_void_p()
    st = lib.qc_eloc_create(h.ctypes.data_as(ctypes.c_void_p), eri.ctypes.data_as(ctypes.c_void_p),
                            float(e_core), int(n_orb), int(n_elec), int(precision), int(mode),
                            ctypes.byref(out))
    _check(st, None)
    buf = torch.zeros(ctypes.sizeof(qc_eloc_summary), dtype=torch.uint8, pin_memory=True)
    return QcHandle(out, n_orb, n_elec, precision, mode, buf)


def qc_eloc_destroy(handle: QcHandle):
    if handle.ptr:
        load_library().qc_eloc_destroy(handle.ptr)
        handle.ptr = ctypes.c_void_p()


def qc_eloc_reserve(handle: QcHandle, n_u_max: int, n_table_max: int = 0):
    _check(load_library().qc_eloc_reserve(handle.ptr, int(n_u_max), int(n_table_max)), handle.ptr)


def qc_eloc_set_option(handle: QcHandle, option: int, value: int):
    _check(load_library().qc_eloc_set_option(handle.ptr, int(option), int(value)), handle.ptr)


def qc_eloc_pairs_per_sample(handle: QcHandle) -> int:
    return int(load_library().qc_eloc_pairs_per_sample(handle.ptr))


def qc_eloc_timings(handle: QcHandle):
    ms = (ctypes.c_float * 3)()
    _check(load_library().qc_eloc_timings(handle.ptr, ms), handle.ptr)
    return tuple(float(v) for v in ms)


def qc_eloc_last_config(handle: QcHandle) -> dict:
    c = (ctypes.c_int64 * 7)()
    _check(load_library().qc_eloc_last_config(handle.ptr, c), handle.ptr)
    return dict(kernel=int(c[0]), grid=int(c[1]), warps=int(c[2]), unroll=int(c[3]), smem=int(c[4]),
                filter_log2w=int(c[5]), chunks=int(c[6]))


def qc_test_fail_alloc(after: int):
    """Test hook: the library's next `after` device allocations succeed, the one after fails
    as out-of-memory (negative: off)."""
    _check(load_library().qc_test_fail_alloc(int(after)), None)


def qc_eloc_work(handle: QcHandle) -> dict:
    """Work counts of the last evaluation made with QC_OPT_COUNT_WORK = 1 (waits for it)."""
    w = (ctypes.c_uint64 * len(WORK_FIELDS))()
    _check(load_library().qc_eloc_work(handle.ptr, w, len(WORK_FIELDS)), handle.ptr)
    return {k: int(v) for k, v in zip(WORK_FIELDS, w)}


def _dptr(t, name, dtype_ok, shape_last=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype not in dtype_ok:
        raise ValueError(f"{name}: dtype {t.dtype} not in {dtype_ok}")
    if shape_last is not None and (t.dim() != 2 or t.shape[-1] != shape_last):
        raise ValueError(f"{name} must have shape (n, {shape_last})")
    return ctypes.c_void_p(t.data_ptr())


def qc_eloc_eval(handle: QcHandle, samples, counts, psi, table_keys=None, table_psi=None,
                 eloc=None, diagnostics: bool = False, summary: bool = True, stream=None,
                 hit_cursor=None, hit_list=None):
    """Enqueue one evaluation.  Returns (eloc complex128[n_u], diag) where diag is None or
    a dict of per-sample hit_count / hit_rowsum / hit_signsum tensors.  The summary is
    written into ``handle.summary_buf``; read it with ``qc_eloc_summary_read`` after the
    stream has passed the call.  ``hit_cursor`` (int64[n_u], each sample's first position)
    and ``hit_list`` (int64) receive the pair-by-pair lists (qc_eloc_out in the header)."""
    import torch
    lib = load_library()
    key_types = (torch.int64, torch.uint64)
    psi_types = (torch.complex128, torch.float64)
    n_u = samples.shape[0]
    if eloc is None:
        eloc = torch.empty(n_u, dtype=torch.complex128, device=samples.device)
    diag = None
    out = qc_eloc_out()
    out.eloc = eloc.data_ptr()
    out.summary = handle.summary_buf.data_ptr() if summary else None
    if diagnostics:
        diag = dict(hit_count=torch.empty(n_u, dtype=torch.int32, device=samples.device),
                    hit_rowsum=torch.empty(n_u, dtype=torch.int64, device=samples.device),
                    hit_signsum=torch.empty(n_u, dtype=torch.int64, device=samples.device))
        out.hit_count = diag["hit_count"].data_ptr()
        out.hit_rowsum = diag["hit_rowsum"].data_ptr()
        out.hit_signsum = diag["hit_signsum"].data_ptr()
    if (hit_cursor is None) != (hit_list is None):
        raise ValueError("hit_cursor and hit_list go together")
    if hit_list is not None:
        if hit_cursor.numel() < n_u:
            raise ValueError("hit_cursor needs one entry per sample")
        out.hit_cursor = _dptr(hit_cursor, "hit_cursor", (torch.int64,)).value
        out.hit_list = _dptr(hit_list, "hit_list", (torch.int64,)).value
        out.hit_list_cap = int(hit_list.numel())
    s = _dptr(samples, "samples", key_types, 2)
    c = _dptr(counts, "counts", (torch.int64,))
    p = _dptr(psi, "psi", psi_types)
    tk = _dptr(table_keys, "table_keys", key_types, 2)
    tp = _dptr(table_psi, "table_psi", psi_types)
    n_t = 0 if table_keys is None else table_keys.shape[0]
    if stream is None:
        stream = torch.cuda.current_stream(samples.device)
    st = lib.qc_eloc_eval(handle.ptr, s, c, p, int(n_u), tk, tp, int(n_t), ctypes.byref(out),
                          ctypes.c_void_p(stream.cuda_stream))
    _check(st, handle.ptr)
    return eloc, diag


def qc_eloc_grad(handle: QcHandle, eloc, counts, dconj=None, weights: bool = True, stream=None):
    """Eq. 4 on the device after the handle's last evaluation (same stream): returns
    (w complex128[n_u] or None, g float64[n_par] or None) with w_i = c_i (E_loc,i - Ebar)/W
    and g_p = 2 Re sum_i w_i dconj[i, p] (dconj: complex128 [n_u, n_par], d ln Psi* rows)."""
    import torch
    lib = load_library()
    n_u = eloc.shape[0]
    e = _dptr(eloc, "eloc", (torch.complex128,))
    c = _dptr(counts, "counts", (torch.int64,))
    d = None
    n_par = 0
    g = None
    if dconj is not None:
        if dconj.dim() != 2 or dconj.shape[0] != n_u:
            raise ValueError("dconj must be [n_u, n_par]")
        d = _dptr(dconj, "dconj", (torch.complex128,))
        n_par = dconj.shape[1]
        g = torch.empty(n_par, dtype=torch.float64, device=eloc.device)
    w = torch.empty(n_u, dtype=torch.complex128, device=eloc.device) if weights else None
    if stream is None:
        stream = torch.cuda.current_stream(eloc.device)
    st = lib.qc_eloc_grad(handle.ptr, e, c, int(n_u), d, int(n_par),
                          None if w is None else ctypes.c_void_p(w.data_ptr()),
                          None if g is None else ctypes.c_void_p(g.data_ptr()),
                          ctypes.c_void_p(stream.cuda_stream))
    _check(st, handle.ptr)
    return w, g


def qc_eloc_export(handle: QcHandle, samples, keys=True, elems=True, diag=True, stream=None):
    """The connected set of every sample in the export order: returns (keys int64[n_u * P, 2]
    or None, elems float64[n_u * P] or None, diag float64[n_u] or None)."""
    import torch
    lib = load_library()
    n_u = samples.shape[0]
    P = qc_eloc_pairs_per_sample(handle)
    dev = samples.device
    k = torch.empty((n_u * P, 2), dtype=torch.int64, device=dev) if keys else None
    e = torch.empty(n_u * P, dtype=torch.float64, device=dev) if elems else None
    d = torch.empty(n_u, dtype=torch.float64, device=dev) if diag else None
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    vp = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    st = lib.qc_eloc_export(handle.ptr, _dptr(samples, "samples", (torch.int64, torch.uint64), 2), int(n_u),
                            vp(k), vp(e), vp(d), ctypes.c_void_p(stream.cuda_stream))
    _check(st, handle.ptr)
    return k, e, d


def qc_eloc_apply(handle: QcHandle, psi, counts, elems, diag, psi_conn, eloc=None, summary: bool = True,
                  stream=None):
    """E_loc against psi on the exported connected set; returns eloc (complex128[n_u]) and
    writes the Eq. 1 summary into handle.summary_buf (read with qc_eloc_summary_read)."""
    import torch
    lib = load_library()
    n_u = psi.shape[0]
    if eloc is None:
        eloc = torch.empty(n_u, dtype=torch.complex128, device=psi.device)
    if stream is None:
        stream = torch.cuda.current_stream(psi.device)
    st = lib.qc_eloc_apply(handle.ptr, _dptr(psi, "psi", (torch.complex128,)), _dptr(counts, "counts", (torch.int64,)),
                           int(n_u), _dptr(elems, "elems", (torch.float64,)), _dptr(diag, "diag", (torch.float64,)),
                           _dptr(psi_conn, "psi_conn", (torch.complex128,)), ctypes.c_void_p(eloc.data_ptr()),
                           ctypes.c_void_p(handle.summary_buf.data_ptr()) if summary else None,
                           ctypes.c_void_p(stream.cuda_stream))
    _check(st, handle.ptr)
    return eloc


def qc_probe_peaks(stream=None) -> dict:
    """Measured ceilings on the current device: {'alu_ops_per_s', 'l2_gather_gbs'}."""
    import torch
    a, g = ctypes.c_double(0.0), ctypes.c_double(0.0)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load_library().qc_probe_peaks(ctypes.byref(a), ctypes.byref(g), ctypes.c_void_p(stream.cuda_stream)), None)
    return dict(alu_ops_per_s=a.value, l2_gather_gbs=g.value)


def qc_dedup_workspace_bytes(n_raw: int) -> int:
    return int(load_library().qc_dedup_workspace_bytes(int(n_raw)))


def qc_dedup(raw, n_orb: int, keys_out=None, counts_out=None, n_unique=None, work=None, stream=None):
    """The sample table of a raw stream on the device: returns (keys_out, counts_out,
    n_unique) tensors -- the first int(n_unique) rows are the table (read n_unique after the
    stream has passed the call; -1 means a key had a bit >= n_orb set)."""
    import torch
    lib = load_library()
    n = raw.shape[0]
    dev = raw.device
    if keys_out is None:
        keys_out = torch.empty((max(n, 1), 2), dtype=torch.int64, device=dev)
    if counts_out is None:
        counts_out = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    if n_unique is None:
        n_unique = torch.empty(1, dtype=torch.int64, device=dev)
    need = qc_dedup_workspace_bytes(n)
    if work is None or work.numel() < need:
        work = torch.empty(need + 256, dtype=torch.uint8, device=dev)
    wp = work.data_ptr()
    wp += (-wp) % 256
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    st = lib.qc_dedup(_dptr(raw, "raw", (torch.int64, torch.uint64), 2) if n else None, int(n), int(n_orb),
                      ctypes.c_void_p(keys_out.data_ptr()), ctypes.c_void_p(counts_out.data_ptr()),
                      ctypes.c_void_p(n_unique.data_ptr()), ctypes.c_void_p(wp), int(need),
                      ctypes.c_void_p(stream.cuda_stream))
    _check(st, None)
    return keys_out, counts_out, n_unique


QC_STATIC_MAX_SAMPLES = 131072


def qc_eloc_eval_static(h, eri, e_core: float, n_orb: int, n_elec: int, samples, counts, psi,
                        eloc, summary=None, stream=None):
    """The allocation-free entry point: every argument is caller-owned memory (h, eri and
    the sample arrays on the device, ``summary`` a page-locked uint8 tensor or None).
    Returns the status code; raises QcError with the library's message on failure."""
    import torch
    lib = load_library()
    K = int(n_orb) // 2
    for name, t, n in (("h", h, K * K), ("eri", eri, K ** 4)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
        if t.numel() < n:
            raise ValueError(f"{name} needs {n} entries for n_orb = {n_orb}")
    n_u = samples.shape[0]
    for name, t in (("counts", counts), ("psi", psi), ("eloc", eloc)):
        if t.shape[0] < n_u:
            raise ValueError(f"{name} has fewer rows than samples ({t.shape[0]} < {n_u})")
    if summary is not None and (summary.is_cuda or summary.numel() < ctypes.sizeof(qc_eloc_summary)):
        raise ValueError("summary must be host memory of at least sizeof(qc_eloc_summary) bytes")
    if stream is None:
        stream = torch.cuda.current_stream(samples.device)
    st = lib.qc_eloc_eval_static(ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(eri.data_ptr()),
                                 float(e_core), int(n_orb), int(n_elec),
                                 _dptr(samples, "samples", (torch.int64, torch.uint64), 2),
                                 _dptr(counts, "counts", (torch.int64,)),
                                 _dptr(psi, "psi", (torch.complex128, torch.float64)), int(n_u),
                                 _dptr(eloc, "eloc", (torch.complex128,)),
                                 None if summary is None else ctypes.c_void_p(summary.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))
    if st != QC_OK:
        raise QcError(st, lib.qc_eloc_last_error(None).decode())
    return st


def qc_eloc_summary_read(handle: QcHandle, stream=None) -> dict:
    """Synchronize the stream and return the last summary as a dict."""
    import torch
    (stream or torch.cuda.current_stream()).synchronize()
    return handle.summary_struct().as_dict()


def keys_to_tensor(keys: np.ndarray, device="cuda"):
    """uint64[n, 2] numpy keys -> int64 CUDA tensor with the same bits."""
    import torch
    k = np.ascontiguousarray(keys, dtype=np.uint64).view(np.int64)
    return torch.from_numpy(k).to(device)


# ----------------------------------------------------------------------------------
# the batched form
# ----------------------------------------------------------------------------------
@dataclass
class QcBatch:
    ptr: ctypes.c_void_p
    n_mol: int
    summary_buf: object  # page-locked uint8 tensor, one qc_eloc_summary per molecule
    keep: list           # handles and tensors that must outlive the batch's use


def _bcheck(st, batch):
    if st != QC_OK:
        raise QcError(st, load_library().qc_batch_last_error(batch.ptr if batch else None).decode())


def qc_batch_create(handles) -> QcBatch:
    import torch
    lib = load_library()
    arr = (ctypes.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    out = ctypes.c_void_p()
    st = lib.qc_batch_create(arr, len(handles), ctypes.byref(out))
    if st != QC_OK:
        raise QcError(st, "qc_batch_create failed")
    buf = torch.zeros(len(handles) * ctypes.sizeof(qc_eloc_summary), dtype=torch.uint8, pin_memory=True)
    return QcBatch(out, len(handles), buf, list(handles))


def qc_batch_destroy(batch: QcBatch):
    if batch.ptr:
        load_library().qc_batch_destroy(batch.ptr)
        batch.ptr = ctypes.c_void_p()


def qc_batch_set_inputs(batch: QcBatch, mol: int, samples, counts, psi, eloc):
    import torch
    st = load_library().qc_batch_set_inputs(
        batch.ptr, int(mol), _dptr(samples, "samples", (torch.int64, torch.uint64), 2),
        _dptr(counts, "counts", (torch.int64,)), _dptr(psi, "psi", (torch.complex128, torch.float64)),
        int(samples.shape[0]), _dptr(eloc, "eloc", (torch.complex128, torch.float64)))
    _bcheck(st, batch)
    batch.keep += [samples, counts, psi, eloc]


def qc_batch_set_rows(batch: QcBatch, mol: int, r0: int, r1: int = -1):
    """Evaluate only rows [r0, r1) of molecule `mol` and reduce Eq. 1 over them (a replica's
    piece; the molecule's summary then holds the piece's partials)."""
    _bcheck(load_library().qc_batch_set_rows(batch.ptr, int(mol), int(r0), int(r1)), batch)


def qc_batch_set_config(batch: QcBatch, unroll=0, warps=0, chunk=0):
    _bcheck(load_library().qc_batch_set_config(batch.ptr, int(unroll), int(warps), int(chunk)), batch)


def qc_batch_config(batch: QcBatch) -> dict:
    c = (ctypes.c_int64 * 6)()
    _bcheck(load_library().qc_batch_config(batch.ptr, c), batch)
    return dict(unroll=int(c[0]), warps=int(c[1]), chunk=int(c[2]), grid=int(c[3]),
                molecules=int(c[4]), smem=int(c[5]))


def qc_batch_eval(batch: QcBatch, stream=None):
    import torch
    s = stream or torch.cuda.current_stream()
    _bcheck(load_library().qc_batch_eval(batch.ptr, ctypes.c_void_p(batch.summary_buf.data_ptr()),
                                         ctypes.c_void_p(s.cuda_stream)), batch)


def qc_batch_graph_launch(batch: QcBatch, stream):
    _bcheck(load_library().qc_batch_graph_launch(batch.ptr, ctypes.c_void_p(batch.summary_buf.data_ptr()),
                                                 ctypes.c_void_p(stream.cuda_stream)), batch)


def qc_batch_summaries(batch: QcBatch, stream=None) -> list:
    import torch
    (stream or torch.cuda.current_stream()).synchronize()
    base = batch.summary_buf.data_ptr()
    sz = ctypes.sizeof(qc_eloc_summary)
    return [qc_eloc_summary.from_address(base + m * sz).as_dict() for m in range(batch.n_mol)]


def qc_batch_timings(batch: QcBatch):
    ms = (ctypes.c_float * 3)()
    _bcheck(load_library().qc_batch_timings(batch.ptr, ms), batch)
    return tuple(float(v) for v in ms)


def qc_batch_autotune(batch: QcBatch, stream=None, iters: int = 2):
    import torch
    s = stream or torch.cuda.current_stream()
    best = (ctypes.c_int64 * 4)()
    _bcheck(load_library().qc_batch_autotune(batch.ptr, ctypes.c_void_p(s.cuda_stream), int(iters), best), batch)
    return dict(unroll=int(best[0]), warps=int(best[1]), chunk=int(best[2]), chunk_pairs=int(best[3]))


def qc_batch_set_chunk_pairs(batch: QcBatch, chunk_pairs: int):
    _bcheck(load_library().qc_batch_set_chunk_pairs(batch.ptr, int(chunk_pairs)), batch)


# ----------------------------------------------------------------------------------
# the serving form
# ----------------------------------------------------------------------------------
class qc_eloc_job(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("eri", ctypes.c_void_p), ("e_core", ctypes.c_double),
                ("n_orb", ctypes.c_int), ("n_elec", ctypes.c_int), ("precision", ctypes.c_int),
                ("flags", ctypes.c_int), ("mol_key", ctypes.c_uint64), ("samples", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("psi", ctypes.c_void_p), ("n_u", ctypes.c_int64),
                ("eloc_out", ctypes.c_void_p)]


class qc_eloc_result(ctypes.Structure):
    _fields_ = [("summary", qc_eloc_summary), ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


@dataclass
class QcServer:
    ptr: ctypes.c_void_p
    keep: dict  # ticket -> host arrays that must outlive the request


def _server_lib():
    lib = load_library()
    if not getattr(lib, "_qc_server_typed", False):
        P = ctypes.c_void_p
        lib.qc_server_create.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)]
        lib.qc_eloc_submit.argtypes = [P, ctypes.POINTER(qc_eloc_job), ctypes.POINTER(ctypes.c_uint64)]
        lib.qc_eloc_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(qc_eloc_result), ctypes.c_int]
        lib.qc_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
        lib.qc_server_destroy.argtypes = [P]
        lib.qc_server_set_option.argtypes = [P, ctypes.c_int, ctypes.c_int64]
        for f in ("qc_server_create", "qc_eloc_submit", "qc_eloc_poll", "qc_server_stats", "qc_server_destroy",
                  "qc_server_set_option"):
            getattr(lib, f).restype = ctypes.c_int
        lib._qc_server_typed = True
    return lib


def qc_server_create(device: int = 0, budget_bytes: int = 160 << 30, max_slots: int = 64,
                     n_streams: int = 2) -> QcServer:
    out = ctypes.c_void_p()
    st = _server_lib().qc_server_create(int(device), int(budget_bytes), int(max_slots), int(n_streams),
                                        ctypes.byref(out))
    if st != QC_OK:
        raise QcError(st, "qc_server_create failed")
    return QcServer(out, {})


QC_JOB_BORROW_INTEGRALS = 1


def qc_eloc_submit(server: QcServer, h, eri, e_core: float, n_orb: int, n_elec: int, keys, counts, psi,
                   precision: int = QC_FP64, mol_key: int = 0, want_eloc: bool = True,
                   borrow_integrals: bool = False) -> int:
    """Queue one request (host numpy inputs); returns its ticket.  With borrow_integrals the
    server reads h and eri when it admits the request instead of copying them at submit (they
    are kept alive here until the ticket is polled)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty(len(keys), dtype=np.complex128) if want_eloc else None
    j = qc_eloc_job(h=h.ctypes.data, eri=eri.ctypes.data, e_core=float(e_core), n_orb=int(n_orb),
                    n_elec=int(n_elec), precision=int(precision),
                    flags=QC_JOB_BORROW_INTEGRALS if borrow_integrals else 0, mol_key=int(mol_key),
                    samples=keys.ctypes.data, counts=counts.ctypes.data, psi=psi.ctypes.data, n_u=len(keys),
                    eloc_out=None if out is None else out.ctypes.data)
    t = ctypes.c_uint64()
    st = _server_lib().qc_eloc_submit(server.ptr, ctypes.byref(j), ctypes.byref(t))
    if st != QC_OK:
        raise QcError(st, "qc_eloc_submit refused the request")
    server.keep[t.value] = (keys, counts, psi, out, h, eri)
    return t.value


def qc_eloc_poll(server: QcServer, ticket: int, timeout_us: int = 0):
    """None while pending; else (result dict, E_loc numpy array or None)."""
    r = qc_eloc_result()
    st = _server_lib().qc_eloc_poll(server.ptr, int(ticket), ctypes.byref(r), int(timeout_us))
    if st == QC_PENDING:
        return None
    if st != QC_OK:
        raise QcError(st, "qc_eloc_poll")
    arrays = server.keep.pop(ticket)
    d = r.summary.as_dict()
    d.update(status=r.status, t_submit=r.t_submit, t_admit=r.t_admit, t_start=r.t_start, t_done=r.t_done)
    return d, arrays[3]


def qc_server_stats(server: QcServer) -> dict:
    s = (ctypes.c_uint64 * 4)()
    _server_lib().qc_server_stats(server.ptr, s)
    return dict(bytes_in_use=int(s[0]), in_flight=int(s[1]), waiting=int(s[2]), resident=int(s[3]))


def qc_server_set_option(server: QcServer, option: int, value: int):
    st = _server_lib().qc_server_set_option(server.ptr, int(option), int(value))
    if st != QC_OK:
        raise QcError(st, "qc_server_set_option failed")


def qc_server_destroy(server: QcServer):
    if server.ptr:
        _server_lib().qc_server_destroy(server.ptr)
        server.ptr = ctypes.c_void_p()
