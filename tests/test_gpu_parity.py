"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar (Eq. 5 / Eq. 1): connected sets, table rows and fermionic phases bit-exact, compared
pair by pair (every hit of every sample as phase * (row + 1), written by the kernel where
the hit is resolved, against the oracle's lists); E_loc within 1e-6 relative for the FP64
path; for the FP32-compensated path |Delta E| <= 1e-5 Ha on the count-weighted energy and,
per sample, the forward-error bound of its FP32 terms (``fp32c_bound``).
"""
import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-6     # relative, per-sample E_loc and energy (FP64 path)
ATOL_FP32C = 1e-5    # Ha, count-weighted energy (FP32-compensated path)
U32 = 2.0 ** -24     # unit roundoff of FP32


def fp32c_bound(n_elec, mag):
    """Per-sample bound on |E_loc(FP32-compensated) - E_loc(FP64 oracle)|.  Each term
    <x|H|x'> psi(x')/psi(x) is formed from FP32 integrals and FP32 ratios: the element from at
    most 1 + 3 n_elec / 2 stored integrals summed in FP32 (singles; doubles one or two), each
    stored with relative error <= u, the summation adding at most its length times u of the
    sum of their magnitudes; the ratio from psi(x') and 1/psi(x) rounded to FP32 and a complex
    product (<= 6 u); the term's own product (u); the TwoSum accumulation is exact up to u of
    the lane's sum.  Bounded by (n_elec + 16) u times the oracle's magnitude sum (sum over hits
    of |psi(x')/psi(x)| times the absolute integral terms of the element).  The diagonal and the
    final combination are FP64 (1e-12 relative is left for them)."""
    return (n_elec + 16) * U32 * mag


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23809_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def sort_lists(off, lst):
    """Each sample's entries ordered by table row (the canonical form of a hit set)."""
    n = len(off) - 1
    seg = np.repeat(np.arange(n), np.diff(off))
    return lst[np.lexsort((np.abs(lst), seg))]


def gpu_lists(B, h, kt, ct, pt, tk, tp, hit_count):
    """Pair-by-pair lists of one evaluation: cursors from the hit counts of a previous
    evaluation of the same inputs, then every hit as phase * (row + 1).  Returns (off, sorted
    entries, status); the exit cursors must be exactly the next sample's start."""
    import torch
    cnt = hit_count.to(torch.int64)
    off = torch.zeros(len(cnt) + 1, dtype=torch.int64, device=cnt.device)
    off[1:] = torch.cumsum(cnt, 0)
    cursor = off[:-1].clone()
    lst = torch.full((max(int(off[-1].item()), 1),), 0, dtype=torch.int64, device=cnt.device)
    eloc, _ = B.qc_eloc_eval(h, kt, ct, pt, tk, tp, hit_cursor=cursor, hit_list=lst)
    st = B.qc_eloc_summary_read(h)["status"]
    o = off.cpu().numpy()
    assert np.array_equal(cursor.cpu().numpy(), o[1:]), "a sample's list length differs from its hit count"
    return o, sort_lists(o, lst.cpu().numpy()[:o[-1]]), st, eloc.cpu().numpy()


def run_gpu(B, ints, n_orb, n_elec, keys, counts, psi, table=None, prec=0, mode=0, opts=None,
            diag=True, e_core=0.0, lists=False):
    import torch
    h = B.qc_eloc_create(ints.h, ints.eri, e_core, n_orb, n_elec, prec, mode)
    try:
        for k, v in (opts or {}).items():
            B.qc_eloc_set_option(h, k, v)
        kt = B.keys_to_tensor(keys)
        ct = torch.from_numpy(np.ascontiguousarray(counts, dtype=np.int64)).cuda()
        pt = torch.from_numpy(np.ascontiguousarray(psi, dtype=np.complex128)).cuda()
        tk = tp = None
        if table is not None:
            tk = B.keys_to_tensor(table[0])
            tp = torch.from_numpy(np.ascontiguousarray(table[1], dtype=np.complex128)).cuda()
        eloc, d = B.qc_eloc_eval(h, kt, ct, pt, tk, tp, diagnostics=diag or lists)
        summ = B.qc_eloc_summary_read(h)
        cfg = B.qc_eloc_last_config(h)
        out = dict(eloc=eloc.cpu().numpy(), summary=summ, cfg=cfg)
        if diag or lists:
            out["hits"] = d["hit_count"].cpu().numpy().view(np.uint32)
            out["rowsum"] = d["hit_rowsum"].cpu().numpy().view(np.uint64)
            out["signsum"] = d["hit_signsum"].cpu().numpy()
        if lists:
            out["list_off"], out["list"], st, e2 = gpu_lists(B, h, kt, ct, pt, tk, tp, d["hit_count"])
            assert st == summ["status"]
            # writing the lists leaves the evaluation bitwise unchanged
            assert np.array_equal(e2.view(np.uint64), out["eloc"].view(np.uint64))
        return out
    finally:
        B.qc_eloc_destroy(h)


def assert_sets_equal(g, det, rows=None):
    sel = slice(None) if rows is None else rows
    assert np.array_equal(g["hits"][sel], det["hits"]), "connected sets differ"
    assert np.array_equal(g["rowsum"][sel], det["rowsum"]), "table rows differ"
    assert np.array_equal(g["signsum"][sel], det["signsum"]), "fermionic phases differ"


def assert_lists_equal(g, want, rows=None):
    """Pair by pair: every sample's (row, phase) list equals the oracle's.  want = (off,
    entries) from oracle.hit_lists for the selected rows (all rows when rows is None)."""
    woff, wl = want
    goff, gl = g["list_off"], g["list"]
    if rows is None:
        assert np.array_equal(goff, woff), "hit counts differ"
        assert np.array_equal(gl, wl), "hit lists (rows or phases) differ"
        return
    for k, r in enumerate(rows):
        a = gl[goff[r]:goff[r + 1]]
        b = wl[woff[k]:woff[k + 1]]
        assert np.array_equal(a, b), f"hit list of sample {r} differs"


def assert_eloc_close(got, want, rtol=RTOL_FP64):
    ok = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), ok)
    err = np.abs(got[ok] - want[ok]) / np.maximum(1.0, np.abs(want[ok]))
    assert err.max(initial=0.0) <= rtol, f"max rel err {err.max():.3e}"
    return err.max(initial=0.0)


def assert_fp32c_per_sample(orc, ints, n_orb, n_elec, keys, psi, got, want, table=(None, None), mode=0):
    """Per-sample error of the FP32-compensated path against the FP64 oracle within
    fp32c_bound; returns (|error| per sample, largest error / bound)."""
    mag = orc.magnitudes(ints.h, ints.eri, 0.0, n_orb, keys, psi, table[0], table[1], mode=mode)
    ok = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), ok)
    per = np.abs(got[ok] - want[ok])
    bound = fp32c_bound(n_elec, mag[ok]) + 1e-12 * np.abs(want[ok])
    assert np.all(per <= bound), f"per-sample error {per.max():.3e} above its bound"
    return per, float((per / bound).max(initial=0.0))


KERNELS = [dict(), {2: 1}, {2: 2, 5: 1}, {2: 2, 5: 2}, {2: 2, 5: 4}, {2: 2, 4: 3, 6: 5}, {2: 1, 4: 1, 6: 7},
           {2: 2, 8: 2}, {2: 2, 8: 2, 5: 1}, {2: 2, 10: 1}, {2: 2, 10: 2}, {2: 2, 10: 2, 11: 1},
           {2: 2, 10: 2, 11: 1024}, {2: 2, 10: 2, 8: 2, 5: 1}]


@pytest.mark.parametrize("opts", KERNELS, ids=["auto", "direct", "filt_u1", "filt_u2", "filt_u4",
                                                "filt_w3_g5", "direct_w1_g7", "lean", "lean_u1", "nojoin",
                                                "join", "join_scan", "join_enum", "join_lean_u1"])
def test_tiny_sample_mode(B, orc, opts):
    """N=14, 6 electrons, 1,000 uniform samples (204 pairs each), every kernel variant."""
    ints, s = I.make_workload("n14_e6_u1k")
    g = run_gpu(B, ints, 14, 6, s.keys, s.counts, s.psi, opts=opts, lists=True)
    want, det = orc.eloc(ints.h, ints.eri, 0.0, 14, s.keys, s.psi, details=True)
    assert_sets_equal(g, det)
    assert_lists_equal(g, orc.hit_lists(ints.h, ints.eri, 0.0, 14, s.keys, s.psi))
    assert_eloc_close(g["eloc"], want)
    m, var, w, n = orc.reduce(want, s.counts)
    sm = g["summary"]
    assert sm["status"] == 0 and sm["flags"] == 0
    assert sm["n_pairs"] == 1000 * 204 and sm["n_hits"] == int(det["hits"].sum())
    assert sm["w"] == 100_000 and sm["n_used"] == 1000
    assert abs(sm["energy"] - m) <= RTOL_FP64 * abs(m)
    assert abs(sm["var"] - var) <= RTOL_FP64 * max(1.0, var)
    # the all-pairs scan (no enumeration) finds the same connected set
    assert_lists_equal(g, orc.hit_lists_pairwise(ints.h, ints.eri, 0.0, 14, s.keys, s.psi))


@pytest.mark.parametrize("n,ne,nu,prec", [(76, 20, 3000, 1), (128, 64, 24, 0), (52, 14, 2000, 0)])
def test_lean_lists_equal_stored(B, orc, n, ne, nu, prec):
    """Pair hash lists formed on the fly (QC_OPT_LEAN 2) give the same hashes in the same
    order as the stored lists (QC_OPT_LEAN 1): E_loc bitwise equal, with at least as many
    warps; and both match the oracle."""
    K = n // 2
    ints = I.make_integrals(K, min(n, 52), 990 + n)
    keys = I.rank_weighted_samples(K, ne // 2, ne // 2, nu, seed=991 + n)
    counts = I.zipf_counts(nu, 40 * nu, 992 + n)
    psi = I.lognormal_psi(nu, 993 + n)
    a = run_gpu(B, ints, n, ne, keys, counts, psi, prec=prec, opts={8: 1, 10: 1})
    b = run_gpu(B, ints, n, ne, keys, counts, psi, prec=prec, opts={8: 2, 10: 1}, lists=True)
    assert a["cfg"]["kernel"] == 2 and b["cfg"]["kernel"] == 3
    assert b["cfg"]["warps"] >= a["cfg"]["warps"] and b["cfg"]["filter_log2w"] == a["cfg"]["filter_log2w"]
    assert np.array_equal(a["eloc"].view(np.uint64), b["eloc"].view(np.uint64))
    assert np.array_equal(a["hits"], b["hits"]) and np.array_equal(a["signsum"], b["signsum"])
    want, det = orc.eloc(ints.h, ints.eri, 0.0, n, keys, psi, details=True)
    assert_sets_equal(b, det)
    assert_lists_equal(b, orc.hit_lists(ints.h, ints.eri, 0.0, n, keys, psi))
    if prec == 0:
        assert_eloc_close(b["eloc"], want)


@pytest.mark.parametrize("n,ne,nu,prec,opts", [(52, 14, 3000, 0, {}), (76, 20, 3000, 1, {}),
                                               (52, 14, 3000, 0, {11: 1}), (52, 14, 3000, 0, {11: 64}),
                                               (52, 14, 2000, 0, {11: 1024}),
                                               (76, 20, 2000, 0, {}), (76, 20, 2000, 1, {11: 1}),
                                               (76, 20, 2000, 1, {11: 1024}),
                                               (76, 20, 2000, 1, {8: 2, 5: 2}), (52, 14, 3000, 0, {9: 2000}),
                                               (40, 8, 1500, 0, {}), (128, 64, 24, 0, {}), (128, 40, 200, 1, {}),
                                               (52, 14, 3000, 0, {14: 1, 11: 1024}), (52, 14, 3000, 0, {14: 4}),
                                               (76, 20, 2000, 1, {14: 3, 11: 64}), (76, 20, 2000, 0, {14: 8, 9: 3000}),
                                               (128, 40, 200, 0, {14: 5})],
                         ids=["n52", "n76_fp32c", "n52_scan_all", "n52_enum_more", "n52_enum_most", "n76_fp64",
                              "n76_scan_all", "n76_enum_most", "n76_lean_u2", "n52_chunks", "n40", "n128",
                              "n128_fp32c", "n52_alpha_seg1", "n52_alpha_seg4", "n76_alpha_seg3", "n76_alpha_seg8_chunks",
                              "n128_alpha_seg5"])
def test_join_equals_enumeration(B, orc, n, ne, nu, prec, opts):
    """The sample-space join (QC_OPT_JOIN 2: short row groups scanned, long ones enumerated)
    finds the same connected set with the same rows and phases as plain enumeration
    (QC_OPT_JOIN 1) and as the oracle; E_loc differs only by the order of accumulation.
    Rank-weighted samples give a few very large groups (the reference determinant's
    strings) beside many small ones, so both halves of the join run."""
    K = n // 2
    ints = I.make_integrals(K, min(n, 52), 1990 + n)
    na = (ne + 1) // 2
    keys = I.rank_weighted_samples(K, na, ne - na, nu, seed=1991 + n)
    counts = I.zipf_counts(nu, 40 * nu, 1992 + n)
    psi = I.lognormal_psi(nu, 1993 + n)
    a = run_gpu(B, ints, n, ne, keys, counts, psi, prec=prec, opts={2: 2, 10: 1, **opts}, lists=True)
    b = run_gpu(B, ints, n, ne, keys, counts, psi, prec=prec, opts={2: 2, 10: 2, **opts}, lists=True)
    assert a["cfg"]["kernel"] in (2, 3) and b["cfg"]["kernel"] in (4, 5)
    assert np.array_equal(a["list_off"], b["list_off"]) and np.array_equal(a["list"], b["list"])
    want, det = orc.eloc(ints.h, ints.eri, 0.0, n, keys, psi, details=True)
    assert_sets_equal(b, det)
    assert_lists_equal(b, orc.hit_lists(ints.h, ints.eri, 0.0, n, keys, psi))
    if prec == 0:
        assert_eloc_close(b["eloc"], want)
        assert_eloc_close(b["eloc"], a["eloc"], rtol=1e-12)
    else:
        m, _, _, _ = orc.reduce(want, counts)
        assert abs(b["summary"]["energy"] - m) <= ATOL_FP32C
        assert_fp32c_per_sample(orc, ints, n, ne, keys, psi, b["eloc"], want)
    assert b["summary"]["status"] == 0 and b["summary"]["n_hits"] == a["summary"]["n_hits"]


def test_join_deterministic(B):
    """Two runs of the join path give bitwise-equal E_loc (group order inside the index is
    row order, whatever order the build's atomics took)."""
    K = 26
    ints = I.make_integrals(K, 52, 2052)
    keys = I.rank_weighted_samples(K, 7, 7, 4000, seed=2053)
    counts = I.zipf_counts(4000, 160000, 2054)
    psi = I.lognormal_psi(4000, 2055)
    r = [run_gpu(B, ints, 52, 14, keys, counts, psi, opts={10: 2}, diag=False)["eloc"] for _ in range(2)]
    assert np.array_equal(r[0].view(np.uint64), r[1].view(np.uint64))


@pytest.mark.parametrize("join", [1, 2], ids=["enumeration", "join"])
def test_join_caller_table_and_invalid_row(B, orc, join):
    """Sample-space mode against a caller's table: samples half in the table and half not
    (a sample whose spin strings have no group in the table), with the join forced on and
    off; then a table row with a wrong electron count, which the join index leaves out of
    every group -- the other samples' connected sets and E_loc are unchanged."""
    K = 26
    ints = I.make_integrals(K, 52, 3101)
    allk = I.rank_weighted_samples(K, 7, 7, 5000, seed=3102)
    rng = np.random.default_rng(3103)
    in_tab = np.zeros(len(allk), bool)
    in_tab[rng.choice(len(allk), 3500, replace=False)] = True
    tkeys, tpsi = allk[in_tab], I.lognormal_psi(int(in_tab.sum()), 3104)
    pick = np.sort(np.concatenate([np.flatnonzero(~in_tab)[:700], np.flatnonzero(in_tab)[:700]]))
    skeys = allk[pick]
    spsi = I.lognormal_psi(len(skeys), 3105)
    counts = I.zipf_counts(len(skeys), 50 * len(skeys), 3106)
    g = run_gpu(B, ints, 52, 14, skeys, counts, spsi, table=(tkeys, tpsi), opts={10: join}, lists=True)
    assert g["cfg"]["kernel"] in ((2, 3) if join == 1 else (4, 5))
    want, det = orc.eloc(ints.h, ints.eri, 0.0, 52, skeys, spsi, tkeys, tpsi, details=True)
    assert_sets_equal(g, det)
    assert_lists_equal(g, orc.hit_lists(ints.h, ints.eri, 0.0, 52, skeys, spsi, tkeys, tpsi))
    assert_eloc_close(g["eloc"], want)
    assert g["summary"]["status"] == 0
    # a table row with one electron too many (an empty orbital filled): flagged, in no group
    bad = tkeys.copy()
    r = 1234
    occ = int(bad[r, 0])
    free = next(b for b in range(52) if not (occ >> b) & 1)
    bad[r, 0] = np.uint64(occ | (1 << free))
    order = np.lexsort((bad[:, 0], bad[:, 1]))
    bad, bpsi = bad[order], tpsi[order]
    g2 = run_gpu(B, ints, 52, 14, skeys, counts, spsi, table=(bad, bpsi), opts={10: join}, lists=True)
    assert g2["summary"]["status"] == -4
    want2, det2 = orc.eloc(ints.h, ints.eri, 0.0, 52, skeys, spsi, bad, bpsi, details=True)
    assert_sets_equal(g2, det2)
    # the oracle has no electron-count check of table rows: the bad row's key has no
    # connected sample with the right count, so both lists leave it out
    assert_lists_equal(g2, orc.hit_lists(ints.h, ints.eri, 0.0, 52, skeys, spsi, bad, bpsi))
    assert_eloc_close(g2["eloc"], want2)


def test_reserve_then_eval_allocates_nothing(B):
    """After qc_eloc_reserve, an evaluation within the reserved sizes -- here one that takes
    the sample-space join (20,000 rows) -- allocates no device memory."""
    import torch
    K = 26
    ints = I.make_integrals(K, 52, 3201)
    keys = I.rank_weighted_samples(K, 7, 7, 20000, seed=3202)
    counts = I.zipf_counts(20000, 400000, 3203)
    psi = I.lognormal_psi(20000, 3204)
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 52, 14)
    try:
        kt = B.keys_to_tensor(keys)
        ct = torch.from_numpy(counts).cuda()
        pt = torch.from_numpy(psi).cuda()
        out = torch.empty(len(keys), dtype=torch.complex128, device="cuda")
        B.qc_eloc_reserve(h, len(keys), len(keys))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        B.qc_eloc_eval(h, kt, ct, pt, eloc=out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert B.qc_eloc_last_config(h)["kernel"] in (4, 5)
    finally:
        B.qc_eloc_destroy(h)


def test_exact_ground_state_constant_eloc(B, orc):
    """N=8, 4 electrons, psi = exact ground state of the sector: E_loc = E0 everywhere
    psi is not negligible (FP64 path)."""
    ints = I.make_integrals(4, 8, 808)
    basis = orc.sector(8, 2, 2)
    H = orc.h_definition(ints.h, ints.eri, 0.0, 8, basis)
    w, v = np.linalg.eigh(H)
    psi = v[:, 0].astype(complex) * np.exp(0.3j)
    g = run_gpu(B, ints, 8, 4, basis, np.ones(len(basis), np.int64), psi)
    big = np.abs(psi) > 1e-8 * np.abs(psi).max()
    assert np.abs(g["eloc"][big] - w[0]).max() < 1e-9
    assert np.linalg.norm(g["eloc"] * psi - w[0] * psi) < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_full_mode(B, orc, prec):
    """Accurate energy: a caller table covering every connected x' (the whole sector)."""
    ints = I.make_integrals(6, 12, 61)
    basis = orc.sector(12, 3, 3)
    tpsi = I.lognormal_psi(len(basis), 62)
    rng = np.random.default_rng(63)
    pick = np.sort(rng.choice(len(basis), 120, replace=False))
    keys, psi = basis[pick], tpsi[pick]
    counts = I.multinomial_counts(120, 10_000, 64)
    g = run_gpu(B, ints, 12, 6, keys, counts, psi, table=(basis, tpsi), prec=prec, mode=1, lists=True)
    want, det = orc.eloc(ints.h, ints.eri, 0.0, 12, keys, psi, basis, tpsi, mode=orc.FULL, details=True)
    assert_sets_equal(g, det)
    assert_lists_equal(g, orc.hit_lists(ints.h, ints.eri, 0.0, 12, keys, psi, basis, tpsi, mode=orc.FULL))
    assert np.all(det["hits"] == det["pairs"])
    if prec == 0:
        assert_eloc_close(g["eloc"], want)
    else:
        assert_fp32c_per_sample(orc, ints, 12, 6, keys, psi, g["eloc"], want, (basis, tpsi), mode=orc.FULL)
    m, var, w, n = orc.reduce(want, counts)
    tol = RTOL_FP64 * abs(m) if prec == 0 else ATOL_FP32C
    assert abs(g["summary"]["energy"] - m) <= tol
    assert g["summary"]["status"] == 0


def test_full_mode_reports_missing(B, orc):
    ints = I.make_integrals(5, 10, 71)
    basis = orc.sector(10, 2, 2)
    tpsi = I.lognormal_psi(len(basis), 72)
    keep = np.ones(len(basis), bool)
    keep[[3, 40]] = False
    keys, psi = basis[:30], tpsi[:30]
    g = run_gpu(B, ints, 10, 4, keys, np.ones(30, np.int64), psi, table=(basis[keep], tpsi[keep]), mode=1)
    want = orc.eloc(ints.h, ints.eri, 0.0, 10, keys, psi, basis[keep], tpsi[keep], mode=orc.FULL)
    assert np.array_equal(np.isnan(g["eloc"].real), np.isnan(want.real))
    assert np.isnan(want.real).any()
    sm = g["summary"]
    assert sm["status"] == -9 and sm["n_missing"] > 0 and sm["n_bad"] == int(np.isnan(want.real).sum())


def test_medium_n52_and_shards(B, orc):
    """N=52, 14 electrons, 3,000 rank-weighted samples: full oracle comparison; then two
    shards evaluated against the whole table combine to the same energy."""
    ints = I.make_integrals(26, 52, 5201)
    keys = I.rank_weighted_samples(26, 7, 7, 3000, seed=5202)
    counts = I.zipf_counts(3000, 300_000, 5203)
    psi = I.lognormal_psi(3000, 5204)
    g = run_gpu(B, ints, 52, 14, keys, counts, psi, lists=True)
    want, det = orc.eloc(ints.h, ints.eri, 0.0, 52, keys, psi, details=True)
    assert_sets_equal(g, det)
    assert_lists_equal(g, orc.hit_lists(ints.h, ints.eri, 0.0, 52, keys, psi))
    assert_eloc_close(g["eloc"], want)
    assert g["summary"]["n_pairs"] == 3000 * 25137
    m, var, w, n = orc.reduce(want, counts)
    assert abs(g["summary"]["energy"] - m) <= RTOL_FP64 * abs(m)
    # run-to-run bitwise determinism of every kernel variant and precision
    for opts, prec in (({2: 1}, 0), ({2: 2, 5: 2}, 0), ({}, 1)):
        r1 = run_gpu(B, ints, 52, 14, keys, counts, psi, opts=opts, prec=prec)
        r2 = run_gpu(B, ints, 52, 14, keys, counts, psi, opts=opts, prec=prec)
        assert np.array_equal(r1["eloc"].view(np.uint64), r2["eloc"].view(np.uint64)), (opts, prec)
        assert_sets_equal(r1, det)
    parts = []
    for lo, hi in ((0, 1234), (1234, 3000)):
        gs = run_gpu(B, ints, 52, 14, keys[lo:hi], counts[lo:hi], psi[lo:hi], table=(keys, psi))
        assert_sets_equal(gs, {k: v[lo:hi] for k, v in det.items()})
        assert_eloc_close(gs["eloc"], want[lo:hi])
        parts.append(gs["summary"])
    W = sum(p["w"] for p in parts)
    E = sum(complex(p["sum_ce_re"], p["sum_ce_im"]) for p in parts) / W
    assert W == w and abs(E - m) <= RTOL_FP64 * abs(m)


def test_join_shards_equal_the_whole_bitwise(B, orc):
    """With the sample-space join, rows evaluated against a caller's table (two shards of the
    sample set, each ordered heavy first by its groups looked up in the table's sets) give
    bitwise the E_loc of the same rows in one evaluation of the whole set (ordered by the
    table's own group sizes): the order schedules samples, it never changes a sample's sum."""
    ints = I.make_integrals(26, 52, 5301)
    keys = I.rank_weighted_samples(26, 7, 7, 4000, seed=5302)
    counts = I.zipf_counts(4000, 400_000, 5303)
    psi = I.lognormal_psi(4000, 5304)
    whole = run_gpu(B, ints, 52, 14, keys, counts, psi, opts={10: 2}, diag=False)
    assert whole["cfg"]["kernel"] in (4, 5)
    for lo, hi in ((0, 1500), (1500, 4000)):
        gs = run_gpu(B, ints, 52, 14, keys[lo:hi], counts[lo:hi], psi[lo:hi], table=(keys, psi), opts={10: 2},
                     diag=False)
        # the same kernel form and shape; the grid follows the rows and never enters a sum
        assert {k: v for k, v in gs["cfg"].items() if k != "grid"} == \
            {k: v for k, v in whole["cfg"].items() if k != "grid"}
        assert np.array_equal(gs["eloc"].view(np.uint64), whole["eloc"][lo:hi].view(np.uint64)), (lo, hi)
    want = orc.eloc(ints.h, ints.eri, 0.0, 52, keys[:300], psi[:300], keys, psi)
    assert_eloc_close(whole["eloc"][:300], want)


def test_full_size_n52_sampled(B, orc):
    """The benchmark workload (N=52, 14 e, 1e5 samples, Zipf counts summing to 1e7) in the
    launch configuration the benchmark uses: 512 sampled rows checked against the oracle
    (which looks x' up in the whole table), plus exact structural totals and run-to-run
    determinism."""
    ints, s = I.make_workload("n52_e14_u100k")
    g = run_gpu(B, ints, 52, 14, s.keys, s.counts, s.psi, lists=True)
    g2 = run_gpu(B, ints, 52, 14, s.keys, s.counts, s.psi)
    assert g["cfg"]["kernel"] in (4, 5)
    assert np.array_equal(g["eloc"].view(np.uint64), g2["eloc"].view(np.uint64))
    rows = np.sort(np.random.default_rng(7).choice(s.n_u, 512, replace=False))
    want, det = orc.eloc(ints.h, ints.eri, 0.0, 52, s.keys[rows], s.psi[rows], s.keys, s.psi, details=True)
    assert_sets_equal(g, det, rows)
    assert_lists_equal(g, orc.hit_lists(ints.h, ints.eri, 0.0, 52, s.keys[rows], s.psi[rows], s.keys, s.psi), rows)
    assert_eloc_close(g["eloc"][rows], want)
    sm = g["summary"]
    assert sm["n_pairs"] == 100_000 * 25137 and sm["w"] == 10_000_000 and sm["status"] == 0
    # the energy of the GPU E_loc array reduced by the oracle's reduction
    m, var, w, n = orc.reduce(g["eloc"], s.counts)
    assert abs(sm["energy"] - m) <= 1e-12 * abs(m) and abs(sm["var"] - var) <= 1e-10 * var


def test_beta_phase_same_set_n52(B, orc):
    """The join's beta' phase (for a sample with many alpha' groups too long to scan, a beta'
    group is scanned for the rows of those groups instead of enumerating the beta' against
    each of them; in the launches with a capped alpha list, here 132 of the 133 slots) finds
    the same connected set: at the N=52 workload every sample's hit list with the phase
    equals its list without it, pair by pair, 256 sampled rows equal the oracle's, and E_loc
    agrees to rounding (only the order of accumulation differs)."""
    ints, s = I.make_workload("n52_e14_u100k")
    seg = {B.QC_OPT_ALPHA_SLOTS: 7 * 19 - 1}
    on = run_gpu(B, ints, 52, 14, s.keys, s.counts, s.psi, lists=True, diag=False, opts=seg)
    off = run_gpu(B, ints, 52, 14, s.keys, s.counts, s.psi, lists=True, diag=False,
                  opts={**seg, B.QC_OPT_BETA_COST: -1})
    rows = np.sort(np.random.default_rng(52).choice(s.n_u, 256, replace=False))
    assert_lists_equal(on, orc.hit_lists(ints.h, ints.eri, 0.0, 52, s.keys[rows], s.psi[rows], s.keys, s.psi), rows)
    assert on["cfg"] == off["cfg"] and on["cfg"]["kernel"] in (4, 5)
    assert np.array_equal(on["list_off"], off["list_off"]), "hit counts differ"
    assert np.array_equal(on["list"], off["list"]), "hit lists differ"
    err = np.abs(on["eloc"] - off["eloc"]) / np.maximum(1.0, np.abs(off["eloc"]))
    assert err.max() <= 1e-12, f"max rel difference {err.max():.3e}"


@pytest.mark.parametrize("prec,slots", [(0, 132), (1, 132), (0, 8), (1, 8)])
def test_beta_phase_forced(B, orc, prec, slots):
    """The beta' phase on most samples of a 20,000-row N=52 table (join on, groups judged long
    at a quarter of the default length, every beta' group of up to 4 x the long alpha' groups
    scanned; 132 alpha slots, or 8, where the phase follows the first of several alpha-list
    segments): the hit
    lists of all rows equal those of the filtered enumeration without the join, and 300
    sampled rows equal the oracle's."""
    K = 26
    ints = I.make_integrals(K, 52, 5401)
    keys = I.rank_weighted_samples(K, 7, 7, 20000, seed=5402)
    counts = I.zipf_counts(20000, 200_000, 5403)
    psi = I.lognormal_psi(20000, 5404)
    forced = {B.QC_OPT_JOIN: 2, B.QC_OPT_SCAN_COST: 16, B.QC_OPT_BETA_COST: 1, B.QC_OPT_ALPHA_SLOTS: slots}
    a = run_gpu(B, ints, 52, 14, keys, counts, psi, prec=prec, lists=True, diag=False, opts=forced)
    b = run_gpu(B, ints, 52, 14, keys, counts, psi, prec=prec, lists=True, diag=False, opts={B.QC_OPT_JOIN: 1})
    assert a["cfg"]["kernel"] in (4, 5) and b["cfg"]["kernel"] in (2, 3)
    assert np.array_equal(a["list_off"], b["list_off"]) and np.array_equal(a["list"], b["list"])
    rows = np.sort(np.random.default_rng(54).choice(20000, 300, replace=False))
    assert_lists_equal(a, orc.hit_lists(ints.h, ints.eri, 0.0, 52, keys[rows], psi[rows], keys, psi), rows)
    if prec == 0:
        want = orc.eloc(ints.h, ints.eri, 0.0, 52, keys[rows], psi[rows], keys, psi)
        assert_eloc_close(a["eloc"][rows], want)


def test_precision_form_n76(B, orc):
    """FP32 integrals and FP32 x FP32 terms with TwoSum accumulation; diagonal and the
    reduction in FP64.  N=76, 20 electrons, 4,000 samples: error against the FP64 oracle
    per sample (reported) and on the total (<= 1e-5 Ha)."""
    ints = I.make_integrals(38, 76, 7601)
    keys = I.rank_weighted_samples(38, 10, 10, 4000, seed=7602)
    counts = I.zipf_counts(4000, 400_000, 7603)
    psi = I.lognormal_psi(4000, 7604)
    g = run_gpu(B, ints, 76, 20, keys, counts, psi, prec=1, lists=True)
    want, det = orc.eloc(ints.h, ints.eri, 0.0, 76, keys, psi, details=True)
    assert_sets_equal(g, det)
    assert_lists_equal(g, orc.hit_lists(ints.h, ints.eri, 0.0, 76, keys, psi))
    m, var, w, n = orc.reduce(want, counts)
    err_total = abs(g["summary"]["energy"] - m)
    per, frac = assert_fp32c_per_sample(orc, ints, 76, 20, keys, psi, g["eloc"], want)
    print(f"FP32-comp N=76: |dE| total {err_total:.2e} Ha, per-sample max {per.max():.2e}, "
          f"rms {np.sqrt((per**2).mean()):.2e}, max error / bound {frac:.3f}")
    assert err_total <= ATOL_FP32C
    assert g["summary"]["n_pairs"] == 4000 * 112980


@pytest.mark.slow
def test_full_size_n76_sampled(B, orc):
    """The precision-form workload at full size (N=76, 20 e, 2e5 samples, FP32 integrals and
    terms, FP64 diagonal and reduction) in its default launch (the sample-space join): the
    hit lists of 512 sampled rows pair by pair against the oracle, every sample's E_loc
    within its FP32 forward-error bound, and the count-weighted energy within 1e-5 Ha of the
    FP64 oracle's over all 2e5 samples."""
    ints, s = I.make_workload("n76_e20_u200k")
    g = run_gpu(B, ints, 76, 20, s.keys, s.counts, s.psi, prec=1, lists=True)
    assert g["cfg"]["kernel"] in (4, 5) and g["summary"]["status"] == 0
    rows = np.sort(np.random.default_rng(76).choice(s.n_u, 512, replace=False))
    assert_lists_equal(g, orc.hit_lists(ints.h, ints.eri, 0.0, 76, s.keys[rows], s.psi[rows], s.keys, s.psi), rows)
    want, mag = orc.eloc_and_magnitudes(ints.h, ints.eri, 0.0, 76, s.keys, s.psi)
    per = np.abs(g["eloc"] - want)
    bound = fp32c_bound(20, mag) + 1e-12 * np.abs(want)
    assert np.all(per <= bound), f"per-sample error {per.max():.3e} above its bound"
    m, var, w, n = orc.reduce(want, s.counts)
    err_total = abs(g["summary"]["energy"] - m)
    print(f"FP32-comp N=76 full size: |dE| total {err_total:.2e} Ha, per-sample max {per.max():.2e}, "
          f"rms {np.sqrt((per ** 2).mean()):.2e}, max error / bound {(per / bound).max():.3f}")
    assert err_total <= ATOL_FP32C
    assert g["summary"]["n_pairs"] == s.n_u * 112980 and g["summary"]["w"] == 20_000_000


@pytest.mark.parametrize("K,ne,n_u", [(2, 2, 4), (64, 4, 300), (64, 64, 24), (20, 20, 500)])
def test_shapes_edge(B, orc, K, ne, n_u):
    """Smallest system (N=4), the largest spin-orbital count (N=128) at low and at half
    filling (1.54 M pairs per sample), and N=40 at half filling."""
    ints = I.make_integrals(K, min(2 * K, 16), 100 + K + ne)
    if K == 2:
        keys = orc.sector(4, 1, 1)
    else:
        keys = I.rank_weighted_samples(K, ne // 2, ne // 2, n_u, seed=200 + K)
    n = len(keys)
    psi = I.lognormal_psi(n, 300 + K)
    counts = I.multinomial_counts(n, 50 * n, 400 + K)
    wl = orc.hit_lists(ints.h, ints.eri, 0.0, 2 * K, keys, psi)
    for opts in ({}, {2: 1}, {2: 2, 10: 2}):
        if 10 in opts and K == 2:
            continue
        g = run_gpu(B, ints, 2 * K, ne, keys, counts, psi, opts=opts, lists=True)
        want, det = orc.eloc(ints.h, ints.eri, 0.0, 2 * K, keys, psi, details=True)
        assert_sets_equal(g, det)
        assert_lists_equal(g, wl)
        assert_eloc_close(g["eloc"], want)


def test_options_out_of_range_refused(B):
    """Every option value outside its documented range is refused with QC_ERR_ARG and leaves
    the handle usable; the documented ends of the ranges are accepted."""
    ints = I.make_integrals(8, 16, 4401)
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 16, 8)
    try:
        bad = [(B.QC_OPT_UNROLL, 3), (B.QC_OPT_LEAN, 3), (B.QC_OPT_JOIN, 3), (B.QC_OPT_JOIN, -1),
               (B.QC_OPT_SCAN_COST, -1), (B.QC_OPT_SCAN_COST, 1025), (B.QC_OPT_BETA_COST, -2),
               (B.QC_OPT_BETA_COST, 1025), (B.QC_OPT_ALPHA_SLOTS, -1), (B.QC_OPT_ALPHA_SLOTS, 4097),
               (B.QC_OPT_CHUNK_PAIRS, -2), (B.QC_OPT_GRID, -1), (B.QC_OPT_WARPS, 25), (B.QC_OPT_KERNEL, 3),
               (B.QC_OPT_FILTER_LOG2W, 4), (B.QC_OPT_FILTER_LOG2W, 16), (99, 0)]
        for opt, v in bad:
            with pytest.raises(B.QcError) as ei:
                B.qc_eloc_set_option(h, opt, v)
            assert ei.value.status == -1, (opt, v)
        good = [(B.QC_OPT_BETA_COST, -1), (B.QC_OPT_BETA_COST, 0), (B.QC_OPT_BETA_COST, 1024),
                (B.QC_OPT_SCAN_COST, 0), (B.QC_OPT_SCAN_COST, 1024), (B.QC_OPT_ALPHA_SLOTS, 4096),
                (B.QC_OPT_JOIN, 2), (B.QC_OPT_UNROLL, 4), (B.QC_OPT_WARPS, 24), (B.QC_OPT_WARPS, 0)]
        for opt, v in good:
            B.qc_eloc_set_option(h, opt, v)
        # still evaluates, and correctly
        keys = I.rank_weighted_samples(8, 4, 4, 300, seed=4402)
        psi = I.lognormal_psi(300, 4403)
        import torch
        e, _ = B.qc_eloc_eval(h, B.keys_to_tensor(keys), torch.ones(300, dtype=torch.int64, device="cuda"),
                              torch.from_numpy(psi).cuda())
        assert B.qc_eloc_summary_read(h)["status"] == 0 and np.all(np.isfinite(e.cpu().numpy()))
        # more alpha slots than alpha singles is the full list: the join kernel, not a fallback
        assert B.qc_eloc_last_config(h)["kernel"] in (4, 5)
    finally:
        B.qc_eloc_destroy(h)


def test_degenerate_inputs(B, orc):
    import torch
    ints, s = I.make_workload("n14_e6_u1k")
    # n_u = 0
    g = run_gpu(B, ints, 14, 6, s.keys[:0], s.counts[:0], s.psi[:0])
    assert g["eloc"].shape == (0,) and g["summary"]["n_used"] == 0 and g["summary"]["n_pairs"] == 0
    # n_u = 1: no other sample in the table, E_loc = diagonal
    g = run_gpu(B, ints, 14, 6, s.keys[:1], s.counts[:1], s.psi[:1])
    v, _ = orc.slater_condon(ints.h, ints.eri, 0.0, 14, s.keys[0], s.keys[0])
    assert abs(g["eloc"][0] - v) <= 1e-12 * abs(v) and g["hits"][0] == 0
    # e_core shifts every E_loc
    g1 = run_gpu(B, ints, 14, 6, s.keys, s.counts, s.psi, e_core=2.5)
    g0 = run_gpu(B, ints, 14, 6, s.keys, s.counts, s.psi)
    assert np.abs(g1["eloc"] - g0["eloc"] - 2.5).max() < 1e-12
    # psi(x) = 0 -> NaN for that sample, excluded, status QC_ERR_ZERO_PSI
    psi = s.psi.copy()
    psi[5] = 0
    g = run_gpu(B, ints, 14, 6, s.keys, s.counts, psi)
    assert np.isnan(g["eloc"][5].real) and g["summary"]["status"] == -8 and g["summary"]["n_used"] == 999
    # duplicate key
    keys = s.keys.copy()
    keys[11] = keys[10]
    assert run_gpu(B, ints, 14, 6, keys, s.counts, s.psi)["summary"]["status"] == -3
    # unsorted keys
    keys = s.keys.copy()
    keys[[20, 21]] = keys[[21, 20]]
    assert run_gpu(B, ints, 14, 6, keys, s.counts, s.psi)["summary"]["status"] == -2
    # wrong electron count / bits beyond n_orb: sample skipped with NaN
    keys = s.keys.copy()
    keys[-1, 0] |= np.uint64(1) << np.uint64(20)
    g = run_gpu(B, ints, 14, 6, keys, s.counts, s.psi)
    assert g["summary"]["status"] == -4 and np.isnan(g["eloc"][-1].real)
    assert g["summary"]["n_pairs"] == 999 * 204
    # negative count
    c = s.counts.copy()
    c[3] = -1
    assert run_gpu(B, ints, 14, 6, s.keys, c, s.psi)["summary"]["status"] == -12
    # misaligned device pointer is rejected synchronously
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 14, 6)
    try:
        kt = B.keys_to_tensor(s.keys)
        raw = torch.empty(2 * len(s.keys) + 1, dtype=torch.int64, device="cuda")
        mis = raw[1:].view(-1, 2)
        with pytest.raises(B.QcError):
            B.qc_eloc_eval(h, mis, torch.from_numpy(s.counts).cuda(), torch.from_numpy(s.psi).cuda())
        with pytest.raises(B.QcError):   # FULL mode needs a table; this handle is SAMPLE: table psi missing
            B.qc_eloc_eval(h, kt, torch.from_numpy(s.counts).cuda(), torch.from_numpy(s.psi).cuda(), kt, None)
    finally:
        B.qc_eloc_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_excitation_chunks(B, orc, prec):
    """A sample's doubles split over C warps (QC_OPT_CHUNK_PAIRS): the connected sets, rows and
    phases stay bit-exact, E_loc within the parity tolerance of the oracle and of the
    one-warp evaluation, bitwise the same run to run; an invalid sample and a psi(x) = 0
    sample are reported once."""
    ints = I.make_integrals(26, 52, 5401)
    keys = I.rank_weighted_samples(26, 7, 7, 2000, seed=5402)
    counts = I.zipf_counts(2000, 100_000, 5403)
    psi = I.lognormal_psi(2000, 5404)
    psi[11] = 0.0
    bad_keys = keys.copy()
    bad_keys[7, 0] ^= np.uint64(1)             # one electron too many or too few
    order = np.lexsort((bad_keys[:, 0], bad_keys[:, 1]))
    bad_keys, psi_b, counts_b = bad_keys[order], psi[order], counts[order]
    a = run_gpu(B, ints, 52, 14, bad_keys, counts_b, psi_b, prec=prec, opts={9: 4000}, lists=True)
    b = run_gpu(B, ints, 52, 14, bad_keys, counts_b, psi_b, prec=prec, opts={9: 4000})
    one = run_gpu(B, ints, 52, 14, bad_keys, counts_b, psi_b, prec=prec, opts={9: -1})
    assert a["cfg"]["chunks"] == 7 and one["cfg"]["chunks"] == 1
    assert np.array_equal(a["eloc"].view(np.uint64), b["eloc"].view(np.uint64))
    assert np.array_equal(a["hits"], one["hits"]) and np.array_equal(a["signsum"], one["signsum"])
    fin = np.isfinite(one["eloc"])
    assert np.array_equal(np.isfinite(a["eloc"]), fin) and (~fin).sum() == 2
    err = np.abs(a["eloc"][fin] - one["eloc"][fin]) / np.maximum(1.0, np.abs(one["eloc"][fin]))
    assert err.max() <= (1e-12 if prec == 0 else 1e-5)
    sa, so = a["summary"], one["summary"]
    assert sa["n_bad"] == so["n_bad"] == 2 and sa["n_used"] == so["n_used"] == 1998
    assert sa["n_hits"] == so["n_hits"] and sa["n_pairs"] == so["n_pairs"]
    # against the oracle on the valid samples (it does not check electron counts itself)
    want, det = orc.eloc(ints.h, ints.eri, 0.0, 52, bad_keys, psi_b, details=True)
    ok = np.isfinite(want) & fin
    assert np.array_equal(a["hits"][ok], det["hits"][ok]) and np.array_equal(a["signsum"][ok], det["signsum"][ok])
    okr = np.flatnonzero(ok)
    assert_lists_equal(a, orc.hit_lists(ints.h, ints.eri, 0.0, 52, bad_keys[okr], psi_b[okr], bad_keys, psi_b), okr)
    if prec == 0:
        assert_eloc_close(a["eloc"][ok], want[ok])
