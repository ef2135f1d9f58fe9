"""Pins for the CPU oracle: each check compares it with something other than itself
(exact diagonalisation, closed forms, invariants of the Hamiltonian of Eq. 2, brute force).

A plausible mistake in the oracle -- a dropped term of Eq. 2, a wrong fermionic sign, a
transposed integral index, a missing spin delta -- breaks at least one of these.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I


def _so_ints(K, seed, rank=None, zero_eri=False):
    ints = I.make_integrals(K, rank or 2 * K, seed)
    if zero_eri:
        ints.eri[:] = 0.0
    return ints


# ---------------------------------------------------------------------------------------
# matrix elements: two independent derivations of Eq. 2
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("K,na,nb,seed", [(4, 2, 2, 3), (4, 3, 1, 4), (5, 2, 1, 5), (7, 3, 3, 6)])
def test_definition_equals_slater_condon(orc, K, na, nb, seed):
    """Eq. 2 applied operator by operator == Slater-Condon rules, element by element."""
    ints = _so_ints(K, seed)
    basis = orc.sector(2 * K, na, nb)
    HD = orc.h_definition(ints.h, ints.eri, 0.25, 2 * K, basis)
    HS = orc.h_slater_condon(ints.h, ints.eri, 0.25, 2 * K, basis)
    scale = np.abs(HD).max()
    assert np.abs(HD - HS).max() <= 1e-13 * scale
    assert np.abs(HD - HD.T).max() <= 1e-14 * scale       # Hermitian (real symmetric)
    # structural zeros: elements between determinants differing by more than 2 electrons
    for r in range(0, len(basis), max(1, len(basis) // 40)):
        for c in range(len(basis)):
            d = (bin(int(basis[r, 0]) ^ int(basis[c, 0])).count("1")
                 + bin(int(basis[r, 1]) ^ int(basis[c, 1])).count("1"))
            if d > 4:
                assert HD[r, c] == 0.0


def test_sector_dimension_and_order(orc):
    basis = orc.sector(14, 3, 3)
    assert basis.shape[0] == math.comb(7, 3) ** 2 == 1225
    ref = I.sector_keys(7, 3, 3)
    assert np.array_equal(basis, ref)


# ---------------------------------------------------------------------------------------
# spectra: closed forms and invariants
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("K,na,nb", [(4, 2, 2), (5, 3, 2), (6, 2, 3)])
def test_one_body_spectrum_is_sums_of_orbital_energies(orc, K, na, nb):
    """With (pq|rs) = 0 the many-body spectrum is every sum of n_alpha + n_beta orbital
    energies (eigenvalues of h), one alpha and one beta subset each.  Any sign error in a
    single excitation breaks this."""
    ints = _so_ints(K, 11 + K, zero_eri=True)
    eps = np.linalg.eigvalsh(ints.h)
    basis = orc.sector(2 * K, na, nb)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 2 * K, basis)
    got = np.sort(np.linalg.eigvalsh(H))
    want = np.sort([sum(eps[list(a)]) + sum(eps[list(b)])
                    for a in itertools.combinations(range(K), na)
                    for b in itertools.combinations(range(K), nb)])
    assert np.abs(got - want).max() < 1e-10
    HS = orc.h_slater_condon(ints.h, ints.eri, 0.0, 2 * K, basis)
    assert np.abs(np.sort(np.linalg.eigvalsh(HS)) - want).max() < 1e-10


@pytest.mark.parametrize("U,t", [(4.0, 1.0), (1.0, 0.5), (10.0, 2.0)])
def test_hubbard_dimer_closed_form(orc, U, t):
    """Two-site Hubbard model (h = -t off-diagonal, (kk|kk) = U): the Sz=0 two-electron
    spectrum is {0, U, (U +- sqrt(U^2 + 16 t^2))/2}."""
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    basis = orc.sector(4, 1, 1)
    H = orc.h_definition(h, eri, 0.0, 4, basis)
    got = np.sort(np.linalg.eigvalsh(H))
    r = math.sqrt(U * U + 16 * t * t)
    want = np.sort([0.0, U, (U - r) / 2, (U + r) / 2])
    assert np.abs(got - want).max() < 1e-12
    HS = orc.h_slater_condon(h, eri, 0.0, 4, basis)
    assert np.abs(np.sort(np.linalg.eigvalsh(HS)) - want).max() < 1e-12


def test_two_orbital_pair_model_closed_form(orc):
    """Two orbitals of different symmetry, two electrons (the minimal-basis H2 pattern):
    the closed-shell determinants |1a1b> and |2a2b> couple only through the exchange
    integral K12 = (12|21); their block is [[2h11+J11, K12], [K12, 2h22+J22]].  The open
    shell pair splits into the triplet at h11+h22+J12-K12 and the singlet at
    h11+h22+J12+K12."""
    h11, h22 = -1.25, -0.47
    J11, J22, J12, K12 = 0.67, 0.70, 0.66, 0.18
    h = np.diag([h11, h22])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0], eri[1, 1, 1, 1] = J11, J22
    eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = J12
    for p, q, r, s in [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1)]:
        eri[p, q, r, s] = K12
    basis = orc.sector(4, 1, 1)
    H = orc.h_definition(h, eri, 0.0, 4, basis)
    a, b = 2 * h11 + J11, 2 * h22 + J22
    closed = [(a + b) / 2 - math.hypot((a - b) / 2, K12), (a + b) / 2 + math.hypot((a - b) / 2, K12)]
    want = np.sort(closed + [h11 + h22 + J12 - K12, h11 + h22 + J12 + K12])
    assert np.abs(np.sort(np.linalg.eigvalsh(H)) - want).max() < 1e-12


@pytest.mark.parametrize("K,na,nb,seed", [(4, 2, 2, 21), (5, 2, 2, 22), (6, 3, 2, 23)])
def test_orbital_rotation_invariance(orc, K, na, nb, seed):
    """The FCI spectrum is invariant under a real orthogonal rotation of the orbitals
    (h -> U^T h U, (pq|rs) rotated on all four indices).  Exercises every double
    excitation and its sign: a wrong phase or a mis-ordered integral index changes the
    spectrum of one of the two Hamiltonians."""
    ints = _so_ints(K, seed)
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(K, K)))
    h2 = Q.T @ ints.h @ Q
    eri2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", ints.eri, Q, Q, Q, Q, optimize=True)
    basis = orc.sector(2 * K, na, nb)
    e1 = np.linalg.eigvalsh(orc.h_definition(ints.h, ints.eri, 0.0, 2 * K, basis))
    e2 = np.linalg.eigvalsh(orc.h_definition(h2, eri2, 0.0, 2 * K, basis))
    assert np.abs(e1 - e2).max() < 1e-9
    e3 = np.linalg.eigvalsh(orc.h_slater_condon(h2, eri2, 0.0, 2 * K, basis))
    assert np.abs(e1 - e3).max() < 1e-9


@pytest.mark.parametrize("K,ne", [(4, 4), (5, 4)])
def test_spin_multiplets(orc, K, ne):
    """H commutes with total spin: every level of the Sz=1 sector reappears in the Sz=0
    sector (the M=0 member of its multiplet)."""
    ints = _so_ints(K, 31 + K)
    e0 = np.linalg.eigvalsh(orc.h_definition(ints.h, ints.eri, 0.0, 2 * K, orc.sector(2 * K, ne // 2, ne // 2)))
    e1 = np.linalg.eigvalsh(orc.h_definition(ints.h, ints.eri, 0.0, 2 * K, orc.sector(2 * K, ne // 2 + 1, ne // 2 - 1)))
    for v in e1:
        assert np.abs(e0 - v).min() < 1e-9


def test_closed_shell_hartree_fock_energy(orc):
    """<Aufbau|H|Aufbau> = E_core + 2 sum_i h_ii + sum_ij [2 (ii|jj) - (ij|ji)], i, j < o."""
    for K, o, seed in [(7, 3, 41), (26, 7, 42), (38, 10, 43)]:
        ints = I.make_integrals(K, 2 * K, seed)
        x = I.aufbau_key(K, o, o)
        v, ph = orc.slater_condon(ints.h, ints.eri, 1.5, 2 * K, x, x)
        occ = range(o)
        want = 1.5 + 2 * sum(ints.h[i, i] for i in occ) + sum(
            2 * ints.eri[i, i, j, j] - ints.eri[i, j, j, i] for i in occ for j in occ)
        assert ph == 1
        assert abs(v - want) <= 1e-12 * max(1.0, abs(want))


# ---------------------------------------------------------------------------------------
# Eq. 5 -- local energy
# ---------------------------------------------------------------------------------------
def test_exact_eigenstate_has_constant_local_energy(orc):
    """N=8, 4 electrons: with psi the exact ground state of the sector, E_loc(x) = E0 for
    every x with non-negligible amplitude, and E_loc * psi = E0 * psi everywhere."""
    ints = I.make_integrals(4, 8, 808)
    basis = orc.sector(8, 2, 2)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 8, basis)
    w, v = np.linalg.eigh(H)
    for phase in (1.0, np.exp(0.7j)):
        psi = v[:, 0] * phase
        el = orc.eloc(ints.h, ints.eri, 0.0, 8, basis, psi)
        big = np.abs(psi) > 1e-8 * np.abs(psi).max()
        assert np.abs(el[big] - w[0]).max() < 1e-10
        assert np.linalg.norm(el * psi - w[0] * psi) < 1e-10
        elf = orc.eloc(ints.h, ints.eri, 0.0, 8, basis, psi, basis, psi, mode=orc.FULL)
        assert np.abs(elf[big] - w[0]).max() < 1e-10


def _dense_restricted_eloc(H, psi_s, rows):
    """E_loc over a sample subset from a dense H (rows index the sector basis)."""
    Hs = H[np.ix_(rows, rows)]
    off = Hs - np.diag(np.diag(Hs))
    return np.diag(Hs) + (off @ psi_s) / psi_s


def test_sample_space_eloc_equals_dense_restricted_sum(orc):
    """N=14, 6 electrons, 1,000 uniform samples: enumeration + lookup equals the dense
    Eq. 2 Hamiltonian restricted to the sample set, and the all-pairs scan finds the same
    connected set (hits, rows and phases bit-exact)."""
    ints, s = I.make_workload("n14_e6_u1k")
    basis = orc.sector(14, 3, 3)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 14, basis)
    pos = {(int(a), int(b)): i for i, (a, b) in enumerate(basis)}
    rows = np.array([pos[(int(a), int(b))] for a, b in s.keys])
    want = _dense_restricted_eloc(H, s.psi, rows)
    got, det = orc.eloc(ints.h, ints.eri, 0.0, 14, s.keys, s.psi, details=True)
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    assert np.all(det["pairs"] == 204)
    pw, pdet = orc.eloc_pairwise(ints.h, ints.eri, 0.0, 14, s.keys, s.psi, details=True)
    assert np.array_equal(det["hits"], pdet["hits"])
    assert np.array_equal(det["rowsum"], pdet["rowsum"])
    assert np.array_equal(det["signsum"], pdet["signsum"])
    assert np.abs(pw - got).max() <= 1e-12 * np.abs(got).max()
    # hits are exactly the nonzero-degree neighbours found from the dense structure
    conn = np.zeros(len(rows), dtype=np.int64)
    sub = s.keys
    for i in range(len(rows)):
        d = (np.array([bin(int(a) ^ int(sub[i, 0])).count("1") for a in sub[:, 0]])
             + np.array([bin(int(b) ^ int(sub[i, 1])).count("1") for b in sub[:, 1]]))
        conn[i] = np.count_nonzero((d == 2) | (d == 4))
    assert np.array_equal(conn, det["hits"].astype(np.int64))


def test_signs_match_dense_definition(orc):
    """The phase the oracle reports for each hit equals the sign structure of the dense
    definition-path H: H_def[x, y] = phase * |integral combination| is checked through
    the sign-weighted row sum recomputed from H_def with the Slater-Condon magnitude."""
    ints = I.make_integrals(5, 10, 77)
    basis = orc.sector(10, 2, 2)
    HD = orc.h_definition(ints.h, ints.eri, 0.0, 10, basis)
    for r in range(len(basis)):
        for c in range(len(basis)):
            if r == c:
                continue
            v, ph = orc.slater_condon(ints.h, ints.eri, 0.0, 10, basis[r], basis[c])
            if ph == 0:
                assert HD[r, c] == 0.0
            else:
                assert abs(HD[r, c] - v) <= 1e-12


def test_full_sector_sample_equals_full_mode(orc):
    """With the sample set equal to the whole sector, the sample-restricted sum is the
    full sum: SAMPLE mode == FULL mode == (H psi)/psi from the dense definition."""
    ints = I.make_integrals(6, 12, 99)
    basis = orc.sector(12, 3, 2)
    psi = I.lognormal_psi(len(basis), 5)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 12, basis)
    want = (H @ psi) / psi
    a = orc.eloc(ints.h, ints.eri, 0.0, 12, basis, psi)
    b = orc.eloc(ints.h, ints.eri, 0.0, 12, basis, psi, basis, psi, mode=orc.FULL)
    assert np.abs(a - want).max() <= 1e-10 * np.abs(want).max()
    assert np.abs(b - want).max() <= 1e-10 * np.abs(want).max()


def test_full_mode_reports_missing(orc):
    ints = I.make_integrals(4, 8, 5)
    basis = orc.sector(8, 2, 2)
    psi = I.lognormal_psi(len(basis), 6)
    keep = np.ones(len(basis), dtype=bool)
    keep[7] = False
    el = orc.eloc(ints.h, ints.eri, 0.0, 8, basis[:5], psi[:5], basis[keep], psi[keep], mode=orc.FULL)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 8, basis)
    for i in range(5):
        if H[i, 7] != 0.0 or i == 7:
            pass
        d = (bin(int(basis[i, 0]) ^ int(basis[7, 0])).count("1")
             + bin(int(basis[i, 1]) ^ int(basis[7, 1])).count("1"))
        assert np.isnan(el[i]) == (d in (2, 4))


@pytest.mark.parametrize("K,na,nb", [(7, 3, 3), (26, 7, 7), (38, 10, 10), (10, 4, 2), (50, 25, 25)])
def test_connected_count_closed_form(orc, K, na, nb):
    """Pairs per determinant = sum over spins of o v + C(o,2) C(v,2), plus o_a v_a o_b v_b."""
    oa, va, ob, vb = na, K - na, nb, K - nb
    want = (oa * va + ob * vb + math.comb(oa, 2) * math.comb(va, 2)
            + math.comb(ob, 2) * math.comb(vb, 2) + oa * va * ob * vb)
    ints = I.make_integrals(K, 1, 1)
    x = I.aufbau_key(K, na, nb).reshape(1, 2)
    rng = np.random.default_rng(K)
    ka = rng.permutation(K)[:na]
    kb = rng.permutation(K)[:nb]
    oa_m = np.zeros((1, K), bool); oa_m[0, ka] = True
    ob_m = np.zeros((1, K), bool); ob_m[0, kb] = True
    y = I.pack_occupations(oa_m, ob_m)
    for d in (x, y):
        _, det = orc.eloc(ints.h, ints.eri, 0.0, 2 * K, d, np.ones(1, complex), details=True)
        assert int(det["pairs"][0]) == want
    if (K, na) == (26, 7):
        assert want == 25137
    if (K, na) == (38, 10):
        assert want == 112980


def test_connected_union_matches_enumeration(orc):
    ints = I.make_integrals(5, 10, 3)
    basis = orc.sector(10, 2, 2)
    u = orc.connected_union(10, basis[:3])
    # brute force: every sector member within 1 or 2 electron moves of one of the three
    want = set()
    for x in basis[:3]:
        for y in basis:
            d = (bin(int(x[0]) ^ int(y[0])).count("1") + bin(int(x[1]) ^ int(y[1])).count("1"))
            if d in (2, 4):
                want.add((int(y[0]), int(y[1])))
    got = {(int(a), int(b)) for a, b in u}
    assert got == want


# ---------------------------------------------------------------------------------------
# Eq. 1 -- reduction
# ---------------------------------------------------------------------------------------
def test_reduce_closed_forms(orc):
    # constant local energy -> zero variance
    e = np.full(100, -3.25 + 0.5j)
    c = np.arange(1, 101, dtype=np.int64)
    m, var, w, n = orc.reduce(e, c)
    assert m == -3.25 + 0.5j and var == 0.0 and w == 5050.0 and n == 100
    # two-point distribution, equal weights: mean 0, variance 1
    e = np.array([1.0, -1.0] * 50, dtype=complex)
    m, var, w, n = orc.reduce(e, np.full(100, 7, dtype=np.int64))
    assert abs(m) < 1e-15 and abs(var - 1.0) < 1e-15
    # NaN samples are excluded
    e = np.array([1.0, np.nan, 3.0], dtype=complex)
    m, var, w, n = orc.reduce(e, np.array([1, 5, 1], dtype=np.int64))
    assert m == 2.0 and var == 1.0 and w == 2.0 and n == 2


def test_reduce_uniform_psi_equals_mean_of_H(orc):
    """psi = 1 and equal counts over the whole sector: mean E_loc = sum_xy H_xy / dim."""
    ints = I.make_integrals(5, 10, 12)
    basis = orc.sector(10, 2, 2)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 10, basis)
    el = orc.eloc(ints.h, ints.eri, 0.0, 10, basis, np.ones(len(basis), complex))
    m, var, w, n = orc.reduce(el, np.full(len(basis), 3, dtype=np.int64))
    assert abs(m - H.sum() / len(basis)) < 1e-11 * abs(m)
    assert w == 3 * len(basis)
