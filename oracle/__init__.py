"""CPU oracle for the local-energy path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA path never imports it, and it imports
nothing from the CUDA path.

The arithmetic lives in ``qc_oracle.c`` (plain C, FP64, ``-ffp-contract=off``); this
module only compiles it with gcc and marshals numpy arrays through ctypes.  Each
function names the paper passage it follows:

  * ``h_definition``   -- Eq. 2 applied operator by operator (dense H on a basis);
  * ``h_slater_condon``/``slater_condon`` -- Slater-Condon rules (Sec. III-B (ii));
  * ``eloc``           -- Eq. 5 by excitation enumeration + binary search in the table;
  * ``eloc_pairwise``  -- Eq. 5 by an all-pairs scan of the table (no enumeration);
  * ``hit_lists`` / ``hit_lists_pairwise`` -- every hit of every sample as phase * (row + 1),
                          from the enumeration or from the scan, for pair-by-pair parity;
  * ``magnitudes``     -- per sample, the sum over hits of |psi(x')/psi(x)| times the absolute
                          integral terms of <x|H|x'>: the scale of an element's rounding error;
  * ``reduce``         -- Eq. 1 count-weighted mean and variance (two-pass);
  * ``grad``           -- Eq. 4 gradient weights and 2 Re contraction with d ln Psi* rows;
  * ``dedup``          -- the unique-sample table of Sec. IV-C-4 (sorted unique keys with
                          their multiplicities) from a raw stream of sampled bitstrings.

Parity pins: every function is checked in ``tests/test_oracle_pins.py`` against exact
diagonalisation, closed forms and invariants; none is pinned only against itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qc_oracle.c")
_LIB = os.path.join(_HERE, "libqc_oracle.so")
_lib = None

SAMPLE = 0
FULL = 1


def build(force: bool = False) -> str:
    """Compile qc_oracle.c into libqc_oracle.so next to it (gcc, OpenMP, FP64)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_grad.argtypes = [P, P, i64, P, i64, P, P]
    lib.orc_grad.restype = i32
    lib.orc_h_definition.argtypes = [P, P, f64, i32, P, i64, P]
    lib.orc_h_definition.restype = i32
    lib.orc_h_slater_condon.argtypes = [P, P, f64, i32, P, i64, P]
    lib.orc_h_slater_condon.restype = i32
    lib.orc_slater_condon.argtypes = [P, P, f64, i32, P, P, P]
    lib.orc_slater_condon.restype = f64
    lib.orc_eloc.argtypes = [P, P, f64, i32, P, P, i64, P, P, i64, i32, P, P, P, P, P, i32]
    lib.orc_eloc.restype = i64
    lib.orc_pairwise.argtypes = [P, P, f64, i32, P, P, i64, P, P, i64, P, P, P, P, i32]
    lib.orc_pairwise.restype = i64
    lib.orc_eloc_lists.argtypes = [P, P, f64, i32, P, P, i64, P, P, i64, i32, P, P, P, P, i32]
    lib.orc_eloc_lists.restype = i64
    lib.orc_pairwise_lists.argtypes = [P, P, f64, i32, P, P, i64, P, P, i64, P, P, P, i32]
    lib.orc_pairwise_lists.restype = i64
    lib.orc_reduce.argtypes = [P, P, i64, P]
    lib.orc_reduce.restype = i32
    lib.orc_connected_union.argtypes = [i32, P, i64, P, i64]
    lib.orc_connected_union.restype = i64
    lib.orc_sector.argtypes = [i32, i32, i32, P, i64]
    lib.orc_sector.restype = i64
    lib.orc_max_threads.argtypes = []
    lib.orc_max_threads.restype = i32
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _ints(h, eri):
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    return h, eri


def _keys(k):
    return np.ascontiguousarray(k, dtype=np.uint64).reshape(-1, 2)


def _cplx(p):
    return np.ascontiguousarray(p, dtype=np.complex128)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def sector(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Sorted basis of the (n_alpha, n_beta) sector (brute force over 2^K strings)."""
    import math
    K = n_orb // 2
    cap = math.comb(K, n_alpha) * math.comb(K, n_beta)
    out = np.zeros((cap, 2), dtype=np.uint64)
    n = _load().orc_sector(n_orb, n_alpha, n_beta, _p(out), cap)
    if n < 0:
        raise ValueError("sector too large for brute force")
    return out[:n]


def h_definition(h, eri, e_core, n_orb, basis) -> np.ndarray:
    """Dense <row|H|col> by applying Eq. 2 operator by operator."""
    h, eri = _ints(h, eri)
    basis = _keys(basis)
    dim = basis.shape[0]
    H = np.zeros((dim, dim))
    rc = _load().orc_h_definition(_p(h), _p(eri), float(e_core), n_orb, _p(basis), dim, _p(H))
    if rc != 0:
        raise ValueError("basis is not closed under H")
    return H


def h_slater_condon(h, eri, e_core, n_orb, basis) -> np.ndarray:
    """Dense <row|H|col> from the Slater-Condon rules."""
    h, eri = _ints(h, eri)
    basis = _keys(basis)
    dim = basis.shape[0]
    H = np.zeros((dim, dim))
    _load().orc_h_slater_condon(_p(h), _p(eri), float(e_core), n_orb, _p(basis), dim, _p(H))
    return H


def slater_condon(h, eri, e_core, n_orb, bra, ket):
    """(<bra|H|ket>, phase) from the Slater-Condon rules."""
    h, eri = _ints(h, eri)
    b = np.ascontiguousarray(bra, dtype=np.uint64).reshape(2)
    k = np.ascontiguousarray(ket, dtype=np.uint64).reshape(2)
    ph = np.zeros(1, dtype=np.int32)
    v = _load().orc_slater_condon(_p(h), _p(eri), float(e_core), n_orb, _p(b), _p(k), _p(ph))
    return float(v), int(ph[0])


def eloc(h, eri, e_core, n_orb, samples, psi, table_keys=None, table_psi=None,
         mode=SAMPLE, nthreads=0, details=False):
    """Eq. 5 by enumeration of every single/double excitation and table lookup.

    Returns E_loc (complex128[n_u]); with ``details`` also a dict of per-sample
    ``pairs``, ``hits``, ``rowsum`` (sum of row+1) and ``signsum`` (sum of phase*(row+1)).
    """
    h, eri = _ints(h, eri)
    samples = _keys(samples)
    psi = _cplx(psi)
    n_u = samples.shape[0]
    if table_keys is not None:
        table_keys = _keys(table_keys)
        table_psi = _cplx(table_psi)
        n_t = table_keys.shape[0]
    else:
        n_t = 0
    out = np.zeros(n_u, dtype=np.complex128)
    pairs = np.zeros(n_u, dtype=np.uint64)
    hits = np.zeros(n_u, dtype=np.uint32)
    rows = np.zeros(n_u, dtype=np.uint64)
    signs = np.zeros(n_u, dtype=np.int64)
    _load().orc_eloc(_p(h), _p(eri), float(e_core), n_orb, _p(samples), _p(psi), n_u,
                     _p(table_keys), _p(table_psi), n_t, int(mode), _p(out), _p(pairs),
                     _p(hits), _p(rows), _p(signs), int(nthreads))
    if details:
        return out, dict(pairs=pairs, hits=hits, rowsum=rows, signsum=signs)
    return out


def eloc_pairwise(h, eri, e_core, n_orb, samples, psi, table_keys=None, table_psi=None,
                  nthreads=0, details=False):
    """Eq. 5 by an all-pairs scan of the table (sample-space sum)."""
    h, eri = _ints(h, eri)
    samples = _keys(samples)
    psi = _cplx(psi)
    n_u = samples.shape[0]
    if table_keys is not None:
        table_keys = _keys(table_keys)
        table_psi = _cplx(table_psi)
        n_t = table_keys.shape[0]
    else:
        n_t = 0
    out = np.zeros(n_u, dtype=np.complex128)
    hits = np.zeros(n_u, dtype=np.uint32)
    rows = np.zeros(n_u, dtype=np.uint64)
    signs = np.zeros(n_u, dtype=np.int64)
    _load().orc_pairwise(_p(h), _p(eri), float(e_core), n_orb, _p(samples), _p(psi), n_u,
                         _p(table_keys), _p(table_psi), n_t, _p(out), _p(hits), _p(rows),
                         _p(signs), int(nthreads))
    if details:
        return out, dict(hits=hits, rowsum=rows, signsum=signs)
    return out


def _table(samples, psi, table_keys, table_psi):
    if table_keys is not None:
        table_keys = _keys(table_keys)
        return table_keys, _cplx(table_psi), table_keys.shape[0]
    return None, None, 0


def _sorted_lists(off, lst):
    """Each sample's entries sorted by table row (|entry|): rows are unique within a
    sample, so this is the canonical form of its hit set."""
    n = len(off) - 1
    seg = np.repeat(np.arange(n), np.diff(off))
    order = np.lexsort((np.abs(lst), seg))
    return lst[order]


def hit_lists(h, eri, e_core, n_orb, samples, psi, table_keys=None, table_psi=None,
              mode=SAMPLE, nthreads=0):
    """Every hit of every sample, from the enumeration of Eq. 5: returns (off int64[n_u + 1],
    entries int64[off[-1]]) with sample r's hits at off[r]:off[r + 1] as phase * (row + 1),
    sorted by row.  The phase is that of the ``details`` signsum (<x'| a+ a+ a a |x> with
    the emptied and the filled spin orbitals each in ascending order)."""
    h, eri = _ints(h, eri)
    samples = _keys(samples)
    psi = _cplx(psi)
    _, det = eloc(h, eri, e_core, n_orb, samples, psi, table_keys, table_psi, mode=mode,
                  nthreads=nthreads, details=True)
    off = np.zeros(samples.shape[0] + 1, dtype=np.int64)
    off[1:] = np.cumsum(det["hits"].astype(np.int64))
    lst = np.zeros(max(int(off[-1]), 1), dtype=np.int64)
    tk, tp, n_t = _table(samples, psi, table_keys, table_psi)
    out = np.zeros(samples.shape[0], dtype=np.complex128)
    _load().orc_eloc_lists(_p(h), _p(eri), float(e_core), n_orb, _p(samples), _p(psi), samples.shape[0],
                           _p(tk), _p(tp), n_t, int(mode), _p(out), _p(off), _p(lst), None, int(nthreads))
    return off, _sorted_lists(off, lst[:off[-1]])


def hit_lists_pairwise(h, eri, e_core, n_orb, samples, psi, table_keys=None, table_psi=None,
                       nthreads=0):
    """The same lists from the all-pairs scan of the table (no enumeration)."""
    h, eri = _ints(h, eri)
    samples = _keys(samples)
    psi = _cplx(psi)
    _, det = eloc_pairwise(h, eri, e_core, n_orb, samples, psi, table_keys, table_psi,
                           nthreads=nthreads, details=True)
    off = np.zeros(samples.shape[0] + 1, dtype=np.int64)
    off[1:] = np.cumsum(det["hits"].astype(np.int64))
    lst = np.zeros(max(int(off[-1]), 1), dtype=np.int64)
    tk, tp, n_t = _table(samples, psi, table_keys, table_psi)
    out = np.zeros(samples.shape[0], dtype=np.complex128)
    _load().orc_pairwise_lists(_p(h), _p(eri), float(e_core), n_orb, _p(samples), _p(psi), samples.shape[0],
                               _p(tk), _p(tp), n_t, _p(out), _p(off), _p(lst), int(nthreads))
    return off, _sorted_lists(off, lst[:off[-1]])


def eloc_and_magnitudes(h, eri, e_core, n_orb, samples, psi, table_keys=None, table_psi=None,
                        mode=SAMPLE, nthreads=0):
    """E_loc as ``eloc`` and, from the same pass, per sample the sum over its hits x' of
    |psi(x')/psi(x)| times the sum of the absolute values of the integral terms of <x|H|x'>
    (|h_ai| + sum_j |<aj|ij>| + |<aj|ji>| for a single, |<ab|ij>| + |<ab|ji>| for a double):
    (complex128[n_u], float64[n_u])."""
    h, eri = _ints(h, eri)
    samples = _keys(samples)
    psi = _cplx(psi)
    tk, tp, n_t = _table(samples, psi, table_keys, table_psi)
    out = np.zeros(samples.shape[0], dtype=np.complex128)
    mag = np.zeros(samples.shape[0], dtype=np.float64)
    _load().orc_eloc_lists(_p(h), _p(eri), float(e_core), n_orb, _p(samples), _p(psi), samples.shape[0],
                           _p(tk), _p(tp), n_t, int(mode), _p(out), None, None, _p(mag), int(nthreads))
    return out, mag


def magnitudes(h, eri, e_core, n_orb, samples, psi, table_keys=None, table_psi=None,
               mode=SAMPLE, nthreads=0):
    """The magnitude sums of ``eloc_and_magnitudes`` alone: float64[n_u]."""
    return eloc_and_magnitudes(h, eri, e_core, n_orb, samples, psi, table_keys, table_psi, mode, nthreads)[1]


def reduce(eloc_vals, counts):
    """Eq. 1: (Ebar complex, variance, W, n_used) over finite E_loc."""
    e = _cplx(eloc_vals)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    out = np.zeros(5)
    _load().orc_reduce(_p(e), _p(c), e.shape[0], _p(out))
    return complex(out[0], out[1]), float(out[2]), float(out[3]), int(out[4])


def grad(eloc_vals, counts, dconj=None):
    """Eq. 4: (w, g) with w_i = c_i (E_loc,i - Ebar)/W (complex) and, when the rows
    D_ip = d/d theta_p ln Psi*(n_i) are given (complex, n x P), g_p = 2 Re sum_i w_i D_ip."""
    e = _cplx(eloc_vals)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    n = e.shape[0]
    w = np.zeros(n, dtype=np.complex128)
    g = None
    P = 0
    d = None
    if dconj is not None:
        d = np.ascontiguousarray(dconj, dtype=np.complex128)
        P = d.shape[1]
        g = np.zeros(P)
    st = _load().orc_grad(_p(e), _p(c), n, _p(d) if d is not None else None, P, _p(w),
                          _p(g) if g is not None else None)
    if st != 0:
        raise ValueError("orc_grad failed (no finite E_loc with positive count?)")
    return w, g


def dedup(raw):
    """The sample table (unique sorted keys, multiplicities) of a raw stream of sampled
    bitstrings uint64[n, 2]: a library sort of the 128-bit keys (hi = word 1 first, then
    word 0), then run lengths of equal neighbours -- the plain definition, no other steps."""
    raw = np.ascontiguousarray(raw, dtype=np.uint64).reshape(-1, 2)
    if raw.shape[0] == 0:
        return raw.copy(), np.zeros(0, dtype=np.int64)
    order = np.lexsort((raw[:, 0], raw[:, 1]))      # last key is primary: word 1, then word 0
    srt = raw[order]
    head = np.ones(srt.shape[0], dtype=bool)
    head[1:] = np.any(srt[1:] != srt[:-1], axis=1)
    starts = np.flatnonzero(head)
    counts = np.diff(np.append(starts, srt.shape[0])).astype(np.int64)
    return srt[starts].copy(), counts


def connected_union(n_orb, samples, cap=None) -> np.ndarray:
    """Sorted, deduplicated union of every single/double excitation of the samples."""
    samples = _keys(samples)
    if cap is None:
        K = n_orb // 2
        cap = samples.shape[0] * (2 * K * K + (K * K) ** 2) + 16
        cap = min(cap, 1 << 26)
    out = np.zeros((cap, 2), dtype=np.uint64)
    n = _load().orc_connected_union(n_orb, _p(samples), samples.shape[0], _p(out), cap)
    if n < 0:
        raise ValueError("connected union exceeds capacity")
    return out[:n].copy()
