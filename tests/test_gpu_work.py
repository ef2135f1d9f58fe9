"""The local-energy kernel's work counters (QC_OPT_COUNT_WORK), which the benchmark's roofline
is computed from, checked against exact expectations: hits by kind from the oracle's
pair-by-pair lists, every structural pair probed by the unfiltered kernel and tested by the
filtered one without the prefilter, the join's filter tests, scanned rows and beta' work at
the benchmark workloads' full sizes from the group sizes and the join's rules, and counting
that leaves E_loc bitwise unchanged."""
import math

import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23809_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def _hit_kinds(keys, off, lst, table):
    """(singles, same-spin doubles, opposite-spin doubles) among the listed hits."""
    even = np.uint64(0x5555555555555555)
    seg = np.repeat(np.arange(len(keys)), np.diff(off))
    rows = np.abs(lst) - 1
    x, y = keys[seg], table[rows]
    d = x ^ y
    nd = np.array([bin(int(a)).count("1") + bin(int(b)).count("1") for a, b in d])
    da = np.array([bin(int(a & even)).count("1") + bin(int(b & even)).count("1") for a, b in d])
    single = nd == 2
    same = (nd == 4) & ((da == 4) | (da == 0))
    return int(single.sum()), int(same.sum()), int(((nd == 4) & ~same).sum())


def _run(B, ints, n_orb, n_elec, s, opts, prec=0):
    import torch
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, n_orb, n_elec, prec)
    try:
        for k, v in opts.items():
            B.qc_eloc_set_option(h, k, v)
        kt = B.keys_to_tensor(s.keys)
        ct = torch.from_numpy(s.counts).cuda()
        pt = torch.from_numpy(s.psi).cuda()
        e0, _ = B.qc_eloc_eval(h, kt, ct, pt)
        B.qc_eloc_set_option(h, B.QC_OPT_COUNT_WORK, 1)
        e1, _ = B.qc_eloc_eval(h, kt, ct, pt)
        w = B.qc_eloc_work(h)
        summ = B.qc_eloc_summary_read(h)
        cfg = B.qc_eloc_last_config(h)
        assert np.array_equal(e0.cpu().numpy().view(np.uint64), e1.cpu().numpy().view(np.uint64))
        return w, summ, cfg
    finally:
        B.qc_eloc_destroy(h)


@pytest.mark.parametrize("opts,kind", [({2: 1}, "direct"), ({2: 2, 10: 1, 7: 0}, "filtered_noprefilter"),
                                       ({2: 2, 10: 1}, "filtered"), ({2: 2, 10: 2}, "join"),
                                       ({2: 2, 10: 2, 8: 2}, "join_lean")])
def test_work_counters(B, orc, opts, kind):
    K = 26
    ints = I.make_integrals(K, 52, 6101)
    keys = I.rank_weighted_samples(K, 7, 7, 3000, seed=6102)
    s = I.SampleSet(keys=keys, counts=I.zipf_counts(3000, 30000, 6103), psi=I.lognormal_psi(3000, 6104))
    w, summ, cfg = _run(B, ints, 52, 14, s, opts)
    off, lst = orc.hit_lists(ints.h, ints.eri, 0.0, 52, s.keys, s.psi)
    n1, n2, n3 = _hit_kinds(s.keys, off, lst, s.keys)
    assert (w["hits_single"], w["hits_same"], w["hits_ab"]) == (n1, n2, n3)
    assert n1 + n2 + n3 == summ["n_hits"]
    assert w["samples"] == 3000 and w["ctas"] == cfg["grid"]
    # hits found by the join's scans: none without the join, some but not all with it
    if kind in ("join", "join_lean"):
        assert 0 < w["hits_scanned"] < summ["n_hits"]
    else:
        assert w["hits_scanned"] == 0
    pairs = summ["n_pairs"]
    if kind == "direct":
        assert w["tests"] == 0 and w["probes"] == pairs and w["scan_rows"] == 0
    elif kind == "filtered_noprefilter":
        assert w["tests"] == pairs and w["scan_rows"] == 0 and w["probes"] < pairs
    elif kind == "filtered":
        assert 0 < w["tests"] < pairs and w["scan_rows"] == 0
    else:
        assert cfg["kernel"] in (4, 5)
        assert w["scan_rows"] > 0 and w["tests"] < pairs


def _spin_strings(keys, K, spin):
    """Each key's alpha (spin 0) or beta (spin 1) string as a K-bit integer."""
    out = np.zeros(len(keys), dtype=np.uint64)
    for k in range(K):
        b = 2 * k + spin
        out |= ((keys[:, b // 64] >> np.uint64(b % 64)) & np.uint64(1)) << np.uint64(k)
    return out


def _single_strings(S, K, o):
    """All o (K - o) single excitations of each K-bit string with o bits set."""
    occ = np.stack([((S >> np.uint64(k)) & np.uint64(1)) == 1 for k in range(K)], axis=1)
    oi = np.argsort(~occ, axis=1, kind="stable")[:, :o].astype(np.uint64)
    vi = np.argsort(occ, axis=1, kind="stable")[:, :K - o].astype(np.uint64)
    one = np.uint64(1)
    return np.stack([S ^ (one << oi[:, i]) ^ (one << vi[:, a]) for i in range(o) for a in range(K - o)], axis=1)


def _join_work(keys, K, o, cap, scan_cost=4, beta_cost=8, min_long=8):
    """The join kernel's filter tests, scanned rows, beta' look-ups and scanned beta' groups
    over all samples of an own table, from the group sizes alone (the kernel's rules):
    x's alpha group is scanned unless len x scan_cost > 4 (beta' in the table + same-spin
    beta doubles), its beta group unless len x scan_cost > 4 (alpha doubles); an alpha' group
    is long when len x scan_cost > 4 (beta' in the table + 1), else scanned; with at least
    min_long long alpha' in the first segment of the alpha list (cap slots) and beta_cost > 0,
    each beta' is looked up and its group scanned when len x beta_cost <= 4 (that number).
    Tests: class 0 one per long alpha', class 1 (x's alpha group enumerated) one per beta'
    left in the list, classes 2 and 3 (x's beta / alpha group enumerated) every same-spin
    double, class 4 long alpha' x beta' left."""
    def group_len(X, u, c):
        p = np.minimum(np.searchsorted(u, X), len(u) - 1)
        return np.where(u[p] == X, c[p], 0)
    npair = math.comb(o, 2) * math.comb(K - o, 2)
    A, Bs = _spin_strings(keys, K, 0), _spin_strings(keys, K, 1)
    (ua, ca), (ub, cb) = np.unique(A, return_counts=True), np.unique(Bs, return_counts=True)
    w = dict(tests=0, scan_rows=0, beta_looked=0, beta_groups=0)
    for lo in range(0, len(keys), 20000):
        a, b = A[lo:lo + 20000], Bs[lo:lo + 20000]
        La = group_len(_single_strings(a, K, o), ua, ca)
        Lb = group_len(_single_strings(b, K, o), ub, cb)
        len_a, len_b = group_len(a, ua, ca), group_len(b, ub, cb)
        nb = (Lb > 0).sum(1)
        enum_a = len_a * scan_cost > 4 * (nb + npair)
        enum_b = len_b * scan_cost > 4 * npair
        long_a = La * scan_cost > 4 * (nb + 1)[:, None]
        nla = long_a.sum(1)
        run = (np.minimum(nla, cap) >= min_long) & (nb > 0) & (beta_cost > 0)
        scan_b = (Lb > 0) & (Lb * beta_cost <= 4 * np.minimum(nla, cap)[:, None]) & run[:, None]
        nb_left = nb - scan_b.sum(1)
        w["tests"] += int((nla + np.where(enum_a, nb_left + npair, 0) + np.where(enum_b, npair, 0)
                           + nla * nb_left).sum())
        w["scan_rows"] += int((np.where(enum_a, 0, len_a) + np.where(enum_b, 0, len_b)
                               + np.where(long_a, 0, La).sum(1) + np.where(scan_b, Lb, 0).sum(1)).sum())
        w["beta_looked"] += int(nb[run].sum())
        w["beta_groups"] += int(scan_b.sum())
    return w


def _assert_join_work(w, want):
    for k, v in want.items():
        assert w[k] == v, f"{k}: counted {w[k]}, the rules give {v}"


def test_work_counters_full_size_n52(B):
    """The benchmark workload's counts are deterministic (the same on every run), the hits
    add up to the summary's, and the filter tests, scanned rows and beta' phase work are
    exactly what the join's rules give from the group sizes: the default launch (no
    alpha-list segments, so no beta' phase), a capped alpha list (132 of 133 slots) with the
    phase, and the same with the phase off."""
    ints, s = I.make_workload("n52_e14_u100k")
    w1, s1, _ = _run(B, ints, 52, 14, s, {})
    w2, _, _ = _run(B, ints, 52, 14, s, {})
    assert w1 == w2
    assert w1["hits_single"] + w1["hits_same"] + w1["hits_ab"] == s1["n_hits"]
    assert w1["samples"] == 100_000
    _assert_join_work(w1, _join_work(s.keys, 26, 7, cap=133, beta_cost=0))
    seg = {B.QC_OPT_ALPHA_SLOTS: 7 * 19 - 1}
    w3, s3, _ = _run(B, ints, 52, 14, s, seg)
    want3 = _join_work(s.keys, 26, 7, cap=7 * 19 - 1)
    assert 0 < want3["beta_groups"] < want3["beta_looked"]
    _assert_join_work(w3, want3)
    w4, s4, _ = _run(B, ints, 52, 14, s, {**seg, B.QC_OPT_BETA_COST: -1})
    _assert_join_work(w4, _join_work(s.keys, 26, 7, cap=7 * 19 - 1, beta_cost=0))
    assert s4["n_hits"] == s3["n_hits"] == s1["n_hits"]
    assert w4["tests"] > w3["tests"] and w4["scan_rows"] < w3["scan_rows"]


@pytest.mark.slow
def test_work_counters_full_size_n76(B):
    """The precision-form workload (N=76, 2e5 samples, 64-slot alpha lists with segments and
    the beta' phase): its counted filter tests, scanned rows and beta' work are exactly what
    the join's rules give from the group sizes."""
    ints, s = I.make_workload("n76_e20_u200k")
    w, sm, cfg = _run(B, ints, 76, 20, s, {B.QC_OPT_ALPHA_SLOTS: 64}, prec=1)
    assert cfg["kernel"] in (4, 5) and sm["status"] == 0
    _assert_join_work(w, _join_work(s.keys, 38, 10, cap=64))
