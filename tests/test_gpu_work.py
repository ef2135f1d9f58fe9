"""The local-energy kernel's work counters (QC_OPT_COUNT_WORK), which the benchmark's roofline
is computed from, checked against exact expectations: hits by kind from the oracle's
pair-by-pair lists, every structural pair probed by the unfiltered kernel and tested by the
filtered one without the prefilter, the join's filter tests, scanned rows and beta' work at
the benchmark workloads' full sizes from the group sizes and the join's rules, and counting
that leaves E_loc bitwise unchanged."""
import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

from join_model import join_work as _join_work

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
