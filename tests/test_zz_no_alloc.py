"""The allocation-free entry point, qc_eloc_eval_static, against qc_eloc_eval and the oracle.

qc_eloc_eval_static serves callers that cannot allocate device memory when they call
(inside a restrictive stream capture, under a framework's own memory pool, or in a loop
that must not wait on the allocator): it keeps its working memory in one device array
owned by the library.  This file is collected last so that a failure here cannot hide
the results of the other tests; it passes alone and after them.
"""
import ctypes

import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL = 1e-6  # the FP64 tolerance of the parity tests


def _workload(n_u, seed):
    ints = I.make_integrals(26, 52, 5201)
    keys = I.rank_weighted_samples(26, 7, 7, n_u, seed=seed)
    counts = I.zipf_counts(n_u, 100 * n_u, seed + 1)
    psi = I.lognormal_psi(n_u, seed + 2)
    return ints, keys, counts, psi


def _handle_eval(B, ints, kt, ct, pt):
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 52, 14)
    try:
        ref, _ = B.qc_eloc_eval(h, kt, ct, pt)
        return ref.cpu().numpy(), B.qc_eloc_summary_read(h)
    finally:
        B.qc_eloc_destroy(h)


def test_static_entry_point_matches_eval_twice(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    build.build()
    B.load_library()
    size = ctypes.sizeof(B.qc_eloc_summary)
    big = _workload(20_000, 5210)
    small = _workload(3_000, 5310)
    ints = big[0]
    hd = torch.from_numpy(ints.h).cuda()
    ed = torch.from_numpy(ints.eri).cuda()
    cases = []
    for _, keys, counts, psi in (big, small):
        kt = B.keys_to_tensor(keys)
        ct = torch.from_numpy(counts).cuda()
        pt = torch.from_numpy(psi).cuda()
        ref, ref_sum = _handle_eval(B, ints, kt, ct, pt)
        out = torch.empty(len(keys), dtype=torch.complex128, device="cuda")
        summ = torch.zeros(size, dtype=torch.uint8).pin_memory()
        cases.append((keys, psi, kt, ct, pt, ref, ref_sum, out, summ))
    # the first call on the device does the set-up; later calls allocate nothing
    B.qc_eloc_eval_static(hd, ed, 0.0, 52, 14, *cases[0][2:5], cases[0][7], cases[0][8])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # two calls in a row on the larger set, then one on a smaller set after it (the scratch
    # keeps what the larger call left: the smaller one must not see it)
    for call, k in enumerate((0, 0, 1)):
        keys, psi, kt, ct, pt, ref, ref_sum, out, summ = cases[k]
        out.fill_(complex("nan"))
        B.qc_eloc_eval_static(hd, ed, 0.0, 52, 14, kt, ct, pt, out, summ)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, f"call {call} allocated device memory"
        got = out.cpu().numpy()
        err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() <= RTOL, f"call {call}: max rel err {err.max():.3e} against qc_eloc_eval"
        sm = B.qc_eloc_summary.from_address(summ.data_ptr()).as_dict()
        assert sm["status"] == 0
        assert sm["n_pairs"] == ref_sum["n_pairs"] and sm["n_hits"] == ref_sum["n_hits"]
        assert abs(sm["energy"] - ref_sum["energy"]) <= RTOL * abs(ref_sum["energy"])
        # sampled rows against the CPU oracle (each looked up in the whole sample table)
        rows = np.sort(np.random.default_rng(call).choice(len(keys), 200, replace=False))
        want = orc.eloc(ints.h, ints.eri, 0.0, 52, keys[rows], psi[rows], keys, psi)
        e2 = np.abs(got[rows] - want) / np.maximum(1.0, np.abs(want))
        assert e2.max() <= RTOL, f"call {call}: max rel err {e2.max():.3e} against the oracle"
    # sizes beyond the compiled maximum are refused before any device work
    n = B.QC_STATIC_MAX_SAMPLES + 1
    with pytest.raises(B.QcError) as ex:
        fake = torch.empty((n, 2), dtype=torch.int64, device="cuda")
        B.qc_eloc_eval_static(hd, ed, 0.0, 52, 14, fake, torch.empty(n, dtype=torch.int64, device="cuda"),
                              torch.empty(n, dtype=torch.complex128, device="cuda"),
                              torch.empty(n, dtype=torch.complex128, device="cuda"))
    assert ex.value.status == -11 and "QC_STATIC_MAX_SAMPLES" in str(ex.value)
    # an output shorter than the sample set is refused by the binding
    keys, psi, kt, ct, pt = cases[1][:5]
    with pytest.raises(ValueError):
        B.qc_eloc_eval_static(hd, ed, 0.0, 52, 14, kt, ct, pt,
                              torch.empty(len(keys) - 1, dtype=torch.complex128, device="cuda"))
