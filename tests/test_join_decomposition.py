"""The decomposition behind the sample-space join (Eq. 5 with x' restricted to the sample set).

For a sample x = (alpha, beta) the connected table rows x' = (alpha', beta') are exactly:
  * rows with alpha' = alpha whose beta strings differ from beta in 2 or 4 orbitals
    (beta singles and beta-beta doubles),
  * rows with beta' = beta whose alpha strings differ from alpha in 4 orbitals
    (alpha-alpha doubles),
  * rows whose alpha' is a single excitation of alpha and whose beta strings differ from beta
    in 0 or 2 orbitals (the alpha single and the alpha-beta doubles),
and these three sets are disjoint.  Checked here against brute force -- every pair of keys
with the same electron count whose occupations differ in one or two electrons -- on seeded
sample sets with the structure of the benchmark's (rank-weighted, a few large groups) and
uniform ones.  The CUDA kernels implement this decomposition; their connected sets are
compared with the oracle's in the GPU parity tests.
"""
import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I


def _strings(keys, K):
    a = np.zeros(len(keys), np.uint64)
    b = np.zeros(len(keys), np.uint64)
    for k in range(K):
        a |= ((keys[:, (2 * k) // 64] >> np.uint64((2 * k) % 64)) & np.uint64(1)) << np.uint64(k)
        b |= ((keys[:, (2 * k + 1) // 64] >> np.uint64((2 * k + 1) % 64)) & np.uint64(1)) << np.uint64(k)
    return [int(v) for v in a], [int(v) for v in b]


def _pc(v):
    return bin(v).count("1")


def _brute(A, Bs):
    """Connected pairs: total excitation degree 1 or 2 (half the popcount of the difference)."""
    n = len(A)
    out = [set() for _ in range(n)]
    for i in range(n):
        for j in range(n):
            if i != j and _pc(A[i] ^ A[j]) + _pc(Bs[i] ^ Bs[j]) in (2, 4):
                out[i].add(j)
    return out


def _join(A, Bs, K):
    ga, gb = {}, {}
    for r, (a, b) in enumerate(zip(A, Bs)):
        ga.setdefault(a, []).append(r)
        gb.setdefault(b, []).append(r)
    out = []
    for a, b in zip(A, Bs):
        found = []
        found += [r for r in ga[a] if _pc(Bs[r] ^ b) in (2, 4)]          # x's alpha group
        found += [r for r in gb[b] if _pc(A[r] ^ a) == 4]               # x's beta group
        occ = [k for k in range(K) if a >> k & 1]
        vir = [k for k in range(K) if not a >> k & 1]
        for i in occ:                                                  # alpha' groups
            for v in vir:
                found += [r for r in ga.get(a ^ (1 << i) ^ (1 << v), []) if _pc(Bs[r] ^ b) in (0, 2)]
        assert len(found) == len(set(found)), "the three kinds of groups overlap"
        out.append(set(found))
    return out


@pytest.mark.parametrize("K,na,nb,n,kind,seed", [(10, 3, 3, 400, "rank", 11), (12, 4, 3, 500, "rank", 12),
                                                 (8, 2, 2, 300, "uniform", 13), (9, 4, 4, 350, "uniform", 14)])
def test_join_groups_give_the_connected_set(K, na, nb, n, kind, seed):
    if kind == "rank":
        keys = I.rank_weighted_samples(K, na, nb, n, seed=seed)
    else:
        keys = I.uniform_samples(K, na, nb, n, seed)
    A, Bs = _strings(keys, K)
    want = _brute(A, Bs)
    got = _join(A, Bs, K)
    assert got == want
    assert sum(len(s) for s in want) > 0
