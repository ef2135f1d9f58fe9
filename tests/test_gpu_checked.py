"""The bounds-checked build (libqc_eloc_checked.so, QC_CHECKED) against the product build.

In the checked build every table, integral and work-list index the kernels form is tested
against its array's length; one out of range sets QC_FLAG_BOUNDS and the call's status
becomes QC_ERR_BOUNDS.  The same evaluations run in two child processes, one per library
(a process loads one of them): every kernel form must report status 0 with no bounds flag
in the checked build, and E_loc must be bitwise the same in both builds (the checks change
no arithmetic) and agree with the oracle.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAG_BOUNDS = 0x200
RTOL = 1e-6

# (name, spatial orbitals, electrons, unique samples, options, precision); options by number:
# 2 kernel, 8 lean, 10 join, 14 alpha-list slots
CASES = [
    ("n8_direct", 16, 8, 1500, {2: 1}, 0),
    ("n8_filtered", 16, 8, 1500, {2: 2, 10: 1}, 0),
    ("n8_join", 16, 8, 1500, {2: 2, 10: 2}, 0),
    ("n8_join_lean", 16, 8, 1500, {2: 2, 10: 2, 8: 2}, 0),
    ("n8_join_fp32c", 16, 8, 1500, {2: 2, 10: 2}, 1),
    ("n14_auto", 26, 14, 3000, {}, 0),
    ("n14_join_seg32", 26, 14, 3000, {2: 2, 10: 2, 14: 32}, 0),
    ("n14_join_seg32_fp32c", 26, 14, 3000, {2: 2, 10: 2, 14: 32}, 1),
    ("n14_filtered_lean", 26, 14, 3000, {2: 2, 10: 1, 8: 2}, 0),
]


def _inputs(K, ne, n_u, seed):
    ints = I.make_integrals(K, min(2 * K, 52), seed)
    keys = I.rank_weighted_samples(K, ne // 2, ne // 2, n_u, seed=seed + 1)
    counts = I.zipf_counts(n_u, 20 * n_u, seed + 2)
    psi = I.lognormal_psi(n_u, seed + 3)
    return ints, keys, counts, psi


def _child(lib_path, out_path):
    """Every case through one library; E_loc, status and flags to an .npz."""
    import torch
    from paper_2506_23809_gb300 import binding as B
    B.load_library(lib_path)
    res = {}
    for i, (name, K, ne, n_u, opts, prec) in enumerate(CASES):
        ints, keys, counts, psi = _inputs(K, ne, n_u, 7100 + 10 * i)
        h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 2 * K, ne, prec)
        try:
            for k, v in opts.items():
                B.qc_eloc_set_option(h, k, v)
            kt = B.keys_to_tensor(keys)
            ct = torch.from_numpy(counts).cuda()
            pt = torch.from_numpy(psi).cuda()
            e, _ = B.qc_eloc_eval(h, kt, ct, pt, diagnostics=True)
            sm = B.qc_eloc_summary_read(h)
            res[name] = e.cpu().numpy()
            res[name + ":st"] = np.array([sm["status"], sm["flags"], B.qc_eloc_last_config(h)["kernel"]])
        finally:
            B.qc_eloc_destroy(h)
    # the batched kernels: an N=8 and an N=14 molecule, the second one as a row piece
    mols = [_inputs(16, 8, 1500, 7300), _inputs(26, 14, 3000, 7310)]
    hs = [B.qc_eloc_create(m[0].h, m[0].eri, 0.0, 2 * K, ne) for m, (K, ne) in zip(mols, ((16, 8), (26, 14)))]
    keep = []
    try:
        b = B.qc_batch_create(hs)
        try:
            for m, (ints, keys, counts, psi) in enumerate(mols):
                t = (B.keys_to_tensor(keys), torch.from_numpy(counts).cuda(), torch.from_numpy(psi).cuda(),
                     torch.full((len(keys),), complex("nan"), dtype=torch.complex128, device="cuda"))
                keep.append(t)
                B.qc_batch_set_inputs(b, m, *t)
            B.qc_batch_set_rows(b, 1, 500, 2500)
            B.qc_batch_eval(b)
            sums = B.qc_batch_summaries(b)
            for m in range(2):
                res[f"batch{m}"] = keep[m][3].cpu().numpy()
                res[f"batch{m}:st"] = np.array([sums[m]["status"], sums[m]["flags"], 0])
        finally:
            B.qc_batch_destroy(b)
    finally:
        for h in hs:
            B.qc_eloc_destroy(h)
    # the allocation-free entry point
    ints, keys, counts, psi = _inputs(26, 14, 3000, 7320)
    summ = torch.zeros(__import__("ctypes").sizeof(B.qc_eloc_summary), dtype=torch.uint8).pin_memory()
    out = torch.empty(len(keys), dtype=torch.complex128, device="cuda")
    B.qc_eloc_eval_static(torch.from_numpy(ints.h).cuda(), torch.from_numpy(ints.eri).cuda(), 0.0, 52, 14,
                          B.keys_to_tensor(keys), torch.from_numpy(counts).cuda(), torch.from_numpy(psi).cuda(),
                          out, summ)
    torch.cuda.synchronize()
    sm = B.qc_eloc_summary.from_address(summ.data_ptr()).as_dict()
    res["static"] = out.cpu().numpy()
    res["static:st"] = np.array([sm["status"], sm["flags"], 0])
    np.savez(out_path, **res)


def _run_child(lib_path, out_path):
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), lib_path, out_path], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, f"child on {os.path.basename(lib_path)} failed:\n{r.stdout[-3000:]}\n{r.stderr[-3000:]}"
    return dict(np.load(out_path))


@pytest.mark.gpu
def test_checked_build_matches_product_build(orc, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    build.build()
    build.build(checked=True)
    plain = _run_child(B.LIB_PATH, str(tmp_path / "plain.npz"))
    chk = _run_child(B.LIB_CHECKED_PATH, str(tmp_path / "checked.npz"))
    names = [c[0] for c in CASES] + ["batch0", "batch1", "static"]
    for name in names:
        st, flags, _ = chk[name + ":st"]
        assert st == 0 and not (int(flags) & FLAG_BOUNDS), f"{name}: checked build status {st} flags {flags:#x}"
        assert plain[name + ":st"][0] == 0
        assert np.array_equal(plain[name].view(np.uint64), chk[name].view(np.uint64)), \
            f"{name}: E_loc differs between the checked and the product build"
    # the kernel forms asked for are the ones that ran (join forms 4/5, filtered 2/3, direct 1)
    kinds = {c[0]: int(chk[c[0] + ":st"][2]) for c in CASES}
    assert kinds["n8_direct"] == 1 and kinds["n8_join"] in (4, 5) and kinds["n14_join_seg32"] in (4, 5)
    # and the values are the oracle's (FP64 cases; the FP32-compensated ones are held to
    # their bound in the parity tests)
    for i, (name, K, ne, n_u, opts, prec) in enumerate(CASES):
        if prec != 0:
            continue
        ints, keys, counts, psi = _inputs(K, ne, n_u, 7100 + 10 * i)
        rows = np.sort(np.random.default_rng(i).choice(n_u, 150, replace=False))
        want = orc.eloc(ints.h, ints.eri, 0.0, 2 * K, keys[rows], psi[rows], keys, psi)
        got = chk[name][rows]
        err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
        assert err.max() <= RTOL, f"{name}: max rel err {err.max():.3e} against the oracle"
    # the batch piece evaluated only its rows; the rows outside it were left untouched
    b1 = chk["batch1"]
    assert np.all(np.isnan(b1[:500])) and np.all(np.isnan(b1[2500:])) and np.all(np.isfinite(b1[500:2500]))


if __name__ == "__main__":
    _child(sys.argv[1], sys.argv[2])
