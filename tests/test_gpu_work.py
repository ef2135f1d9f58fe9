"""The local-energy kernel's work counters (QC_OPT_COUNT_WORK), which the benchmark's roofline
is computed from, checked against exact expectations: hits by kind from the oracle's
pair-by-pair lists, every structural pair probed by the unfiltered kernel and tested by the
filtered one without the prefilter, and counting that leaves E_loc bitwise unchanged."""
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


def _beta_phase_counts(keys, K, o, cap, scan_cost=4, beta_cost=8, min_long=8):
    """(beta' looked up, beta' groups scanned) by the join's beta' phase over all samples of
    an own table, from the group sizes: a sample's alpha' group is long when len x scan_cost
    > 4 (beta' in the table + 1); with at least min_long long ones in the first segment of
    the alpha list (cap slots), each of its beta' is looked up and its group scanned when
    len x beta_cost <= 4 (long alpha' groups in that segment)."""
    def group_len(X, u, c):
        p = np.minimum(np.searchsorted(u, X), len(u) - 1)
        return np.where(u[p] == X, c[p], 0)
    A, Bs = _spin_strings(keys, K, 0), _spin_strings(keys, K, 1)
    (ua, ca), (ub, cb) = np.unique(A, return_counts=True), np.unique(Bs, return_counts=True)
    looked = groups = 0
    for lo in range(0, len(keys), 20000):
        La = group_len(_single_strings(A[lo:lo + 20000], K, o), ua, ca)
        Lb = group_len(_single_strings(Bs[lo:lo + 20000], K, o), ub, cb)
        nb = (Lb > 0).sum(1)
        nla = np.minimum((La * scan_cost > 4 * (nb + 1)[:, None]).sum(1), cap)
        run = (nla >= min_long) & (nb > 0)
        looked += int(nb[run].sum())
        groups += int(((Lb > 0) & (Lb * beta_cost <= 4 * nla[:, None]))[run].sum())
    return looked, groups


def test_work_counters_full_size_n52(B):
    """The benchmark workload's counts are deterministic (the same on every run) and the hits
    add up to the summary's; its default launch (no alpha-list segments) has no beta'
    phase, and with a capped alpha list (132 of 133 slots) the phase looks up and scans
    exactly the beta' the group sizes call for (none with the phase off)."""
    ints, s = I.make_workload("n52_e14_u100k")
    w1, s1, _ = _run(B, ints, 52, 14, s, {})
    w2, _, _ = _run(B, ints, 52, 14, s, {})
    assert w1 == w2
    assert w1["hits_single"] + w1["hits_same"] + w1["hits_ab"] == s1["n_hits"]
    assert w1["samples"] == 100_000
    assert w1["beta_looked"] == 0 and w1["beta_groups"] == 0
    seg = {B.QC_OPT_ALPHA_SLOTS: 7 * 19 - 1}
    w3, s3, _ = _run(B, ints, 52, 14, s, seg)
    looked, groups = _beta_phase_counts(s.keys, 26, 7, cap=7 * 19 - 1)
    assert 0 < groups < looked
    assert (w3["beta_looked"], w3["beta_groups"]) == (looked, groups)
    w4, s4, _ = _run(B, ints, 52, 14, s, {**seg, B.QC_OPT_BETA_COST: -1})
    assert w4["beta_looked"] == 0 and w4["beta_groups"] == 0
    assert s4["n_hits"] == s3["n_hits"] == s1["n_hits"]
    assert w4["tests"] > w3["tests"] and w4["scan_rows"] < w3["scan_rows"]
