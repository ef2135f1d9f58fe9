"""Planted-mistake checks: compile a mutated copy of the oracle (in a temp dir, on the
CPU) and show that the pins reject it.  Each mutant is a plausible slip -- a dropped
term, a wrong sign, a swapped index -- and must fail at least one pin."""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "qc_oracle.c")

MUTANTS = {
    # exchange term of <pq||rs> dropped
    "no_exchange": ("return phys_so(ig, p, q, r, s) - phys_so(ig, p, q, s, r);",
                    "return phys_so(ig, p, q, r, s);"),
    # annihilation sign ignored in the definition path
    "no_annihilation_sign": ("    if (!bit_get(d, k)) return 0;\n    if (count_below(d, k) & 1) *sign = -*sign;\n    bit_clr(d, k);",
                             "    if (!bit_get(d, k)) return 0;\n    bit_clr(d, k);"),
    # chemist index order swapped: (pr|qs) -> (pq|rs)
    "swapped_indices": ("return chem(ig, p >> 1, r >> 1, q >> 1, s >> 1);",
                        "return chem(ig, p >> 1, q >> 1, r >> 1, s >> 1);"),
    # second single-excitation phase of a double dropped (Slater-Condon path)
    "double_phase": ("    if (count_between(&mid, lo, hi) & 1) ph = -ph;\n", "\n"),
    # one-body factor of the two-body sum (1/4 -> 1/2)
    "quarter": ("double c = 0.25 * asym_so(", "double c = 0.5 * asym_so("),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    str(path), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_h_definition.argtypes = [P, P, f64, i32, P, i64, P]
    lib.orc_h_slater_condon.argtypes = [P, P, f64, i32, P, i64, P]
    return lib


def _dense(lib, fn, h, eri, n_orb, basis):
    H = np.zeros((len(basis), len(basis)))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    getattr(lib, fn)(p(h), p(eri), 0.0, n_orb, p(basis), len(basis), p(H))
    return H


def _pins_pass(lib, orc):
    """The subset of pins that needs only dense matrices."""
    K = 4
    ints = I.make_integrals(K, 8, 3)
    basis = orc.sector(8, 2, 2)
    HD = _dense(lib, "orc_h_definition", ints.h, ints.eri, 8, basis)
    HS = _dense(lib, "orc_h_slater_condon", ints.h, ints.eri, 8, basis)
    ok = np.abs(HD - HS).max() < 1e-12
    # rotation invariance on both paths
    Q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(K, K)))
    h2 = Q.T @ ints.h @ Q
    eri2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", ints.eri, Q, Q, Q, Q, optimize=True)
    for fn in ("orc_h_definition", "orc_h_slater_condon"):
        e1 = np.linalg.eigvalsh(_dense(lib, fn, ints.h, ints.eri, 8, basis))
        e2 = np.linalg.eigvalsh(_dense(lib, fn, np.ascontiguousarray(h2), np.ascontiguousarray(eri2), 8, basis))
        ok &= np.abs(e1 - e2).max() < 1e-9
    # one-body closed form
    z = np.zeros_like(ints.eri)
    eps = np.linalg.eigvalsh(ints.h)
    want = np.sort([sum(eps[list(a)]) + sum(eps[list(b)]) for a in itertools.combinations(range(K), 2)
                    for b in itertools.combinations(range(K), 2)])
    got = np.sort(np.linalg.eigvalsh(_dense(lib, "orc_h_definition", ints.h, z, 8, basis)))
    ok &= np.abs(got - want).max() < 1e-10
    # closed-shell Hartree-Fock energy on the Slater-Condon diagonal (Coulomb vs exchange)
    HSd = _dense(lib, "orc_h_slater_condon", ints.h, ints.eri, 8, basis)
    ref = I.aufbau_key(K, 2, 2)
    r = int(np.nonzero((basis[:, 0] == ref[0]) & (basis[:, 1] == ref[1]))[0][0])
    hf = 2 * sum(ints.h[i, i] for i in range(2)) + sum(
        2 * ints.eri[i, i, j, j] - ints.eri[i, j, j, i] for i in range(2) for j in range(2))
    ok &= abs(HSd[r, r] - hf) < 1e-12
    # two-orbital pair model on the definition path (J and K enter differently)
    h11, h22, J11, J22, J12, K12 = -1.25, -0.47, 0.67, 0.70, 0.66, 0.18
    h = np.diag([h11, h22])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0], eri[1, 1, 1, 1] = J11, J22
    eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = J12
    for p, q, r_, s in [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1)]:
        eri[p, q, r_, s] = K12
    b2 = orc.sector(4, 1, 1)
    a, b = 2 * h11 + J11, 2 * h22 + J22
    half = np.hypot((a - b) / 2, K12)
    want2 = np.sort([(a + b) / 2 - half, (a + b) / 2 + half, h11 + h22 + J12 - K12, h11 + h22 + J12 + K12])
    got2 = np.sort(np.linalg.eigvalsh(_dense(lib, "orc_h_definition", h, eri, 4, b2)))
    ok &= np.abs(got2 - want2).max() < 1e-12
    return bool(ok)


def test_unmutated_copy_passes(tmp_path, orc):
    lib = _build(tmp_path, "orig", "#include <math.h>", "#include <math.h>")
    assert _pins_pass(lib, orc)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, orc, name):
    old, new = MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    assert not _pins_pass(lib, orc), f"pins did not catch mutant {name}"
