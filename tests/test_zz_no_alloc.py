"""The allocation-free entry point, qc_eloc_eval_static, against qc_eloc_eval.

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


def _workload():
    ints = I.make_integrals(26, 52, 5201)
    keys = I.rank_weighted_samples(26, 7, 7, 20_000, seed=5210)
    counts = I.zipf_counts(20_000, 2_000_000, 5211)
    psi = I.lognormal_psi(20_000, 5212)
    return ints, keys, counts, psi


def test_static_entry_point_matches_eval_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    build.build()
    B.load_library()
    ints, keys, counts, psi = _workload()
    kt = B.keys_to_tensor(keys)
    ct = torch.from_numpy(counts).cuda()
    pt = torch.from_numpy(psi).cuda()
    # reference: the handle-based entry point
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 52, 14)
    try:
        ref, _ = B.qc_eloc_eval(h, kt, ct, pt)
        ref_sum = B.qc_eloc_summary_read(h)
    finally:
        B.qc_eloc_destroy(h)
    ref = ref.cpu().numpy()
    hd = torch.from_numpy(ints.h).cuda()
    ed = torch.from_numpy(ints.eri).cuda()
    size = ctypes.sizeof(B.qc_eloc_summary)
    for call in range(2):
        out = torch.full((len(keys),), complex("nan"), dtype=torch.complex128, device="cuda")
        summ = torch.zeros(size, dtype=torch.uint8).pin_memory()
        B.qc_eloc_eval_static(hd, ed, 0.0, 52, 14, kt, ct, pt, out, summ)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() <= RTOL, f"call {call}: max rel err {err.max():.3e}"
        sm = B.qc_eloc_summary.from_address(summ.data_ptr()).as_dict()
        assert sm["status"] == 0
        assert sm["n_pairs"] == ref_sum["n_pairs"] and sm["n_hits"] == ref_sum["n_hits"]
        assert abs(sm["energy"] - ref_sum["energy"]) <= RTOL * abs(ref_sum["energy"])
    # sizes beyond the compiled maximum are refused before any device work
    big = B.QC_STATIC_MAX_SAMPLES + 1
    with pytest.raises(B.QcError) as ex:
        fake = torch.empty((big, 2), dtype=torch.int64, device="cuda")
        B.qc_eloc_eval_static(hd, ed, 0.0, 52, 14, fake, torch.empty(big, dtype=torch.int64, device="cuda"),
                              torch.empty(big, dtype=torch.complex128, device="cuda"),
                              torch.empty(big, dtype=torch.complex128, device="cuda"))
    assert ex.value.status == -11 and "QC_STATIC_MAX_SAMPLES" in str(ex.value)
