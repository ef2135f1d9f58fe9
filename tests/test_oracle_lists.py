"""Pins for the oracle's pair-by-pair outputs (``hit_lists``, ``hit_lists_pairwise``) and for
the per-sample magnitude sum (``magnitudes``) that scales the precision form's per-sample
error bound.

The lists are checked against two things other than the enumeration that writes them: the
all-pairs scan of the table (a second derivation of the connected set, Eq. 5 over the
sample space), and phases built here operator by operator from the definition of the
creation and annihilation operators of Eq. 2, with rows found by brute force.
"""
import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I


def _bits(key, n_orb):
    lo, hi = int(key[0]), int(key[1])
    v = lo | (hi << 64)
    return [(v >> k) & 1 for k in range(n_orb)]


def _apply(occ, ops):
    """Apply second-quantized operators right to left (ops[-1] first) to an occupation list:
    a_k gives (-1)^(occupied below k) and empties k, a+_k the same sign and fills k.
    Returns (sign, occupation) or (0, None) if the state vanishes."""
    occ = list(occ)
    sign = 1
    for kind, k in reversed(ops):
        below = sum(occ[:k])
        if kind == "a":
            if not occ[k]:
                return 0, None
            occ[k] = 0
        else:
            if occ[k]:
                return 0, None
            occ[k] = 1
        if below % 2:
            sign = -sign
    return sign, occ


def _definition_lists(n_orb, samples, table):
    """Rows by brute force (same electron count per spin, 2 or 4 differing spin orbitals);
    phase <x'| a+_i a+_j a_b a_a |x> (a < b emptied, i < j filled) by operator application."""
    tb = [_bits(t, n_orb) for t in table]
    lists = []
    for x in samples:
        ox = _bits(x, n_orb)
        ent = []
        for r, oy in enumerate(tb):
            diff = [k for k in range(n_orb) if ox[k] != oy[k]]
            if len(diff) not in (2, 4):
                continue
            if sum(oy[0::2]) != sum(ox[0::2]) or sum(oy[1::2]) != sum(ox[1::2]):
                continue
            emptied = sorted(k for k in diff if ox[k])
            filled = sorted(k for k in diff if oy[k])
            ops = [("c", k) for k in filled] + [("a", k) for k in reversed(emptied)]
            sign, occ = _apply(ox, ops)
            assert occ == oy and sign != 0
            ent.append(sign * (r + 1))
        lists.append(sorted(ent, key=abs))
    return lists


def _split(off, lst):
    return [list(lst[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


@pytest.mark.parametrize("K,na,nb,n_u,seed", [(4, 2, 2, 30, 11), (7, 3, 3, 200, 12), (6, 3, 2, 150, 13)])
def test_lists_by_definition(orc, K, na, nb, n_u, seed):
    """Every listed hit's row and phase equal those found by brute force and by applying the
    operators one at a time; no hit is missing."""
    ints = I.make_integrals(K, 2 * K, seed)
    basis = orc.sector(2 * K, na, nb)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(basis), min(n_u, len(basis)), replace=False))
    keys = basis[pick]
    psi = I.lognormal_psi(len(keys), seed + 1)
    off, lst = orc.hit_lists(ints.h, ints.eri, 0.0, 2 * K, keys, psi)
    want = _definition_lists(2 * K, keys, keys)
    assert _split(off, lst) == want


def test_lists_caller_table_by_definition(orc):
    """Samples evaluated against a separate table (half of them absent from it)."""
    K, na, nb = 5, 2, 2
    ints = I.make_integrals(K, 2 * K, 21)
    basis = orc.sector(2 * K, na, nb)
    rng = np.random.default_rng(22)
    tab = np.sort(rng.choice(len(basis), 60, replace=False))
    smp = np.sort(rng.choice(len(basis), 40, replace=False))
    tkeys, tpsi = basis[tab], I.lognormal_psi(60, 23)
    off, lst = orc.hit_lists(ints.h, ints.eri, 0.0, 2 * K, basis[smp], I.lognormal_psi(40, 24), tkeys, tpsi)
    assert _split(off, lst) == _definition_lists(2 * K, basis[smp], tkeys)


@pytest.mark.parametrize("n,ne,n_u,seed", [(20, 6, 800, 31), (28, 8, 600, 32), (40, 12, 400, 33)])
def test_lists_enumeration_equal_scan(orc, n, ne, n_u, seed):
    """Rank-weighted sample sets (many hits near the reference determinant): the
    enumeration's lists equal the all-pairs scan's, entry by entry."""
    K = n // 2
    ints = I.make_integrals(K, n, seed)
    keys = I.rank_weighted_samples(K, ne // 2, ne // 2, n_u, seed=seed + 1)
    psi = I.lognormal_psi(n_u, seed + 2)
    a_off, a = orc.hit_lists(ints.h, ints.eri, 0.0, n, keys, psi)
    b_off, b = orc.hit_lists_pairwise(ints.h, ints.eri, 0.0, n, keys, psi)
    assert a_off[-1] > n_u
    assert np.array_equal(a_off, b_off) and np.array_equal(a, b)
    # the digests of the details output are sums over the same lists
    _, det = orc.eloc(ints.h, ints.eri, 0.0, n, keys, psi, details=True)
    seg = np.repeat(np.arange(n_u), np.diff(a_off))
    assert np.array_equal(np.bincount(seg, minlength=n_u), det["hits"].astype(np.int64))
    assert np.array_equal(np.bincount(seg, weights=np.abs(a).astype(float), minlength=n_u).astype(np.int64),
                          det["rowsum"].astype(np.int64))
    assert np.array_equal(np.bincount(seg, weights=a.astype(float), minlength=n_u).astype(np.int64),
                          det["signsum"])


# ---------------------------------------------------------------------------------------
# magnitudes
# ---------------------------------------------------------------------------------------
def test_magnitudes_bound_the_offdiagonal_sum(orc):
    """Triangle inequality: |E_loc - <x|H|x>| <= magnitude, for every sample."""
    ints, s = I.make_workload("n14_e6_u1k")
    mag = orc.magnitudes(ints.h, ints.eri, 0.0, 14, s.keys, s.psi)
    e = orc.eloc(ints.h, ints.eri, 0.0, 14, s.keys, s.psi)
    ed = np.array([orc.slater_condon(ints.h, ints.eri, 0.0, 14, k, k)[0] for k in s.keys])
    assert np.all(np.abs(e - ed) <= mag * (1 + 1e-12))
    assert np.all(mag > 0)


def test_magnitudes_one_body_closed_form(orc):
    """With (pq|rs) = 0 every connected x' is a single excitation whose element is +-h_ai, so
    the magnitude is sum over hits of |h_ai| |psi(x')/psi(x)|: with psi = 1 on the whole
    sector it equals the row sum of |H| off the diagonal (dense H by the definition path)."""
    K, na, nb = 5, 2, 3
    ints = I.make_integrals(K, 2 * K, 41)
    ints.eri[:] = 0.0
    basis = orc.sector(2 * K, na, nb)
    psi = np.ones(len(basis), dtype=complex)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 2 * K, basis)
    want = np.abs(H).sum(axis=1) - np.abs(np.diag(H))
    mag = orc.magnitudes(ints.h, ints.eri, 0.0, 2 * K, basis, psi)
    assert np.abs(mag - want).max() <= 1e-13 * want.max()


def test_magnitudes_sign_and_scale(orc):
    """Absolute values: flipping the sign of every two-electron integral leaves the
    magnitudes unchanged (while E_loc changes), and scaling both integral sets by 2 doubles
    them exactly."""
    K = 10
    ints = I.make_integrals(K, 2 * K, 51)
    keys = I.rank_weighted_samples(K, 3, 3, 300, seed=52)
    psi = I.lognormal_psi(300, 53)
    m0 = orc.magnitudes(ints.h, ints.eri, 0.0, 2 * K, keys, psi)
    m1 = orc.magnitudes(ints.h, -ints.eri, 0.0, 2 * K, keys, psi)
    m2 = orc.magnitudes(2 * ints.h, 2 * ints.eri, 0.0, 2 * K, keys, psi)
    assert np.array_equal(m0, m1) and np.array_equal(2 * m0, m2)
    e0 = orc.eloc(ints.h, ints.eri, 0.0, 2 * K, keys, psi)
    e1 = orc.eloc(ints.h, -ints.eri, 0.0, 2 * K, keys, psi)
    assert np.abs(e0 - e1).max() > 1e-3
