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

The kernels split the work further -- short groups scanned, the excitations into long ones
enumerated, and (beta' phase) the groups of some beta' = single excitations of beta scanned
for the rows of long alpha' groups instead of enumerating those beta' against them -- and the
second test checks, at the level of sets, that every rule combination finds each connected
row exactly once.
"""
from collections import Counter
from itertools import combinations

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


def _split(A, Bs, K, o, scan_cost, beta_cost, min_long, cap):
    """Each sample's rows as the kernels find them, as a multiset: the scan-or-enumerate rule
    per group (rows x scan_cost / 4 against the excitations replaced), the alpha list capped
    at cap slots (the beta' phase follows its first segment), and the beta' phase (with at
    least min_long long alpha' in that segment, a beta' group is scanned when its rows x
    beta_cost / 4 are at most their number, keeping rows whose alpha group is long and x's beta
    single when class 1 is enumerated; the other beta' stay in the enumerated list).  Filter
    and bucket probe stand as exact membership.  Also returns the work as the kernel counts it:
    rows scanned, excitations filter-tested, beta' looked up and beta' groups scanned."""
    ga, gb = {}, {}
    for r, (a, b) in enumerate(zip(A, Bs)):
        ga.setdefault(a, []).append(r)
        gb.setdefault(b, []).append(r)
    row_of = {(a, b): r for r, (a, b) in enumerate(zip(A, Bs))}

    def singles(s):
        occ = [k for k in range(K) if s >> k & 1]
        vir = [k for k in range(K) if not s >> k & 1]
        return [s ^ (1 << i) ^ (1 << v) for i in occ for v in vir]

    def doubles(s):
        occ = [k for k in range(K) if s >> k & 1]
        vir = [k for k in range(K) if not s >> k & 1]
        return [s ^ (1 << i) ^ (1 << j) ^ (1 << u) ^ (1 << v) for i, j in combinations(occ, 2)
                for u, v in combinations(vir, 2)]

    npairs = (o * (o - 1) // 2) * ((K - o) * (K - o - 1) // 2)
    out = []
    work = Counter()
    for a, b in zip(A, Bs):
        found = Counter()
        bp = [b1 for b1 in singles(b) if b1 in gb]            # the prefiltered beta list
        la, lb = len(ga.get(a, [])), len(gb.get(b, []))
        enum_a = la > 0 and la * scan_cost > 4 * (len(bp) + npairs)
        enum_b = lb > 0 and lb * scan_cost > 4 * npairs
        if la > 0 and not enum_a:                             # x's alpha group scanned
            found.update(r for r in ga[a] if _pc(Bs[r] ^ b) in (2, 4))
            work["scan_rows"] += la
        if lb > 0 and not enum_b:                             # x's beta group scanned
            found.update(r for r in gb[b] if _pc(A[r] ^ a) == 4)
            work["scan_rows"] += lb
        athr = 4 * (len(bp) + 1)
        long_a = []
        for a1 in singles(a):                                 # alpha' groups
            if a1 not in ga:
                continue
            if len(ga[a1]) * scan_cost > athr:
                long_a.append(a1)
            else:
                found.update(r for r in ga[a1] if _pc(Bs[r] ^ b) in (0, 2))
                work["scan_rows"] += len(ga[a1])
        first = min(len(long_a), cap)                         # long alpha' in the first segment
        blist = bp
        if beta_cost > 0 and first >= min_long and bp:        # the beta' phase
            blist = []
            work["beta_looked"] += len(bp)
            for b1 in bp:
                if len(gb[b1]) * beta_cost <= 4 * first:
                    work["beta_groups"] += 1
                    work["scan_rows"] += len(gb[b1])
                    for r in gb[b1]:
                        d = _pc(A[r] ^ a)
                        if (d == 0 and enum_a) or (d == 2 and len(ga[A[r]]) * scan_cost > athr):
                            found[r] += 1
                else:
                    blist.append(b1)
        for a1 in long_a:                                     # class 0 and class 4
            found.update(row_of[k] for k in [(a1, b)] + [(a1, b1) for b1 in blist] if k in row_of)
            work["tests"] += 1 + len(blist)
        if enum_a:                                            # classes 1 and 3
            cands = [(a, b1) for b1 in blist] + [(a, b2) for b2 in doubles(b)]
            found.update(row_of[k] for k in cands if k in row_of)
            work["tests"] += len(cands)
        if enum_b:                                            # class 2
            cands = [(a2, b) for a2 in doubles(a)]
            found.update(row_of[k] for k in cands if k in row_of)
            work["tests"] += len(cands)
        out.append(found)
    return out, work


@pytest.mark.parametrize("scan_cost,beta_cost,min_long,cap", [(4, 8, 8, 10 ** 9), (16, 1, 8, 4), (64, 1, 2, 3),
                                                              (64, 4, 1, 1), (4, 0, 8, 2), (1, 1, 1, 5)])
def test_split_with_beta_phase_finds_each_pair_once(scan_cost, beta_cost, min_long, cap):
    K, o = 10, 3
    keys = I.rank_weighted_samples(K, o, o, 1200, seed=21)
    A, Bs = _strings(keys, K)
    want = _brute(A, Bs)
    got, _ = _split(A, Bs, K, o, scan_cost, beta_cost, min_long, cap)
    for r, (g, w) in enumerate(zip(got, want)):
        assert max(g.values(), default=1) == 1, f"sample {r}: a row found twice"
        assert set(g) == w, f"sample {r}: connected set differs"


@pytest.mark.parametrize("scan_cost,beta_cost,min_long,cap", [(4, 8, 8, 10 ** 9), (16, 1, 8, 4), (64, 1, 2, 3),
                                                              (64, 4, 1, 1), (4, 0, 8, 2), (1, 1, 1, 5)])
def test_work_model_equals_the_rules_row_by_row(scan_cost, beta_cost, min_long, cap):
    """The vectorised model of the join's work from group sizes (which the GPU work-counter
    tests hold the kernel's counters to) equals the row-by-row emulation of the rules above:
    scanned rows, filter tests, beta' look-ups and scanned beta' groups."""
    from join_model import join_work
    K, o = 10, 3
    keys = I.rank_weighted_samples(K, o, o, 1200, seed=21)
    A, Bs = _strings(keys, K)
    _, work = _split(A, Bs, K, o, scan_cost, beta_cost, min_long, cap)
    model = join_work(keys, K, o, cap, scan_cost=scan_cost, beta_cost=beta_cost, min_long=min_long)
    assert model == {k: work[k] for k in ("tests", "scan_rows", "beta_looked", "beta_groups")}
    assert model["tests"] > 0 and model["scan_rows"] > 0
