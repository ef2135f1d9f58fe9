"""The batched form: molecules of different sizes in one persistent launch.

Each molecule's results must be bitwise those of its own single-handle evaluation (the
per-sample arithmetic is shared), and within the parity tolerances of the oracle; the
CUDA-graph replay must not change them, and the autotuned shape only within rounding."""
import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [(14, 6, 300), (20, 8, 500), (28, 10, 800), (40, 12, 600), (52, 14, 400), (64, 16, 250)]


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23809_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def _molecules():
    mols = []
    for k, (n, ne, nu) in enumerate(SHAPES):
        K = n // 2
        ints = I.make_integrals(K, n, 900 + k)
        keys = I.rank_weighted_samples(K, ne // 2, ne // 2, nu, seed=910 + k)
        counts = I.zipf_counts(nu, 50 * nu, 920 + k)
        psi = I.lognormal_psi(nu, 930 + k)
        mols.append((n, ne, ints, keys, counts, psi))
    return mols


def _dev(B, keys, counts, psi):
    import torch
    return (B.keys_to_tensor(keys), torch.from_numpy(counts).cuda(), torch.from_numpy(psi).cuda())


@pytest.mark.parametrize("prec,join", [(0, 1), (1, 1), (0, 2), (1, 2)], ids=["fp64", "fp32c", "fp64_join", "fp32c_join"])
def test_batch_equals_single_and_oracle(B, orc, prec, join):
    """join 2: every molecule takes the sample-space join, in the batch (one shared index)
    as alone; join 1: none does."""
    import torch
    mols = _molecules()
    handles, singles, ins, outs = [], [], [], []
    try:
        for n, ne, ints, keys, counts, psi in mols:
            h = B.qc_eloc_create(ints.h, ints.eri, 0.0, n, ne, prec)
            B.qc_eloc_set_option(h, B.QC_OPT_JOIN, join)
            handles.append(h)
            kt, ct, pt = _dev(B, keys, counts, psi)
            e, _ = B.qc_eloc_eval(h, kt, ct, pt)
            singles.append((e.cpu().numpy(), B.qc_eloc_summary_read(h)))
            ins.append((kt, ct, pt))
            outs.append(torch.full((len(keys),), complex("nan"), dtype=torch.complex128, device="cuda"))
        batch = B.qc_batch_create(handles)
        try:
            for m, (kt, ct, pt) in enumerate(ins):
                B.qc_batch_set_inputs(batch, m, kt, ct, pt, outs[m])
            B.qc_batch_eval(batch)
            sums = B.qc_batch_summaries(batch)
            first = [o.cpu().numpy().copy() for o in outs]
            if join == 2:
                assert all(B.qc_eloc_last_config(h)["kernel"] in (4, 5) for h in handles)
            for m, (e1, s1) in enumerate(singles):
                assert np.array_equal(first[m].view(np.uint64), e1.view(np.uint64)), f"molecule {m}"
                assert sums[m]["n_hits"] == s1["n_hits"] and sums[m]["n_pairs"] == s1["n_pairs"]
                assert sums[m]["e_re"] == s1["e_re"] and sums[m]["status"] == 0
            # against the oracle
            for m, (n, ne, ints, keys, counts, psi) in enumerate(mols):
                want = orc.eloc(ints.h, ints.eri, 0.0, n, keys, psi)
                mm, var, w, nn = orc.reduce(want, counts)
                if prec == 0:
                    err = np.abs(first[m] - want) / np.maximum(1.0, np.abs(want))
                    assert err.max() <= 1e-6
                    assert abs(sums[m]["energy"] - mm) <= 1e-6 * abs(mm)
                else:
                    assert abs(sums[m]["energy"] - mm) <= 1e-5
            # CUDA-graph replay on a side stream, twice
            side = torch.cuda.Stream()
            for rep in range(2):
                for o in outs:
                    o.fill_(complex("nan"))
                side.wait_stream(torch.cuda.current_stream())
                B.qc_batch_graph_launch(batch, side)
                side.synchronize()
                for m in range(len(mols)):
                    assert np.array_equal(outs[m].cpu().numpy().view(np.uint64), first[m].view(np.uint64))
            # autotuned shape: another unroll or filter size finds the hits in another order,
            # so only the summation order differs -- same hit counts, E_loc within rounding
            best = B.qc_batch_autotune(batch, iters=1)
            assert best["unroll"] in (2, 4)
            B.qc_batch_eval(batch)
            tuned = B.qc_batch_summaries(batch)
            for m in range(len(mols)):
                assert tuned[m]["n_hits"] == sums[m]["n_hits"] and tuned[m]["status"] == 0
                o = outs[m].cpu().numpy()
                tol = 1e-12 if prec == 0 else 1e-5
                assert np.max(np.abs(o - first[m]) / np.maximum(1.0, np.abs(first[m]))) <= tol
        finally:
            B.qc_batch_destroy(batch)
    finally:
        for h in handles:
            B.qc_eloc_destroy(h)


def test_batch_excitation_chunks_equal_single(B):
    """With the same excitation-chunk size the batched evaluation stays bitwise equal to the
    handle API for every molecule."""
    import torch
    mols = _molecules()
    handles, singles, ins, outs = [], [], [], []
    try:
        for n, ne, ints, keys, counts, psi in mols:
            h = B.qc_eloc_create(ints.h, ints.eri, 0.0, n, ne, 0)
            B.qc_eloc_set_option(h, 9, 3000)
            handles.append(h)
            kt, ct, pt = _dev(B, keys, counts, psi)
            e, _ = B.qc_eloc_eval(h, kt, ct, pt)
            singles.append((e.cpu().numpy(), B.qc_eloc_summary_read(h), B.qc_eloc_last_config(h)["chunks"]))
            ins.append((kt, ct, pt))
            outs.append(torch.empty(len(keys), dtype=torch.complex128, device="cuda"))
        assert max(c for _, _, c in singles) > 1
        batch = B.qc_batch_create(handles)
        try:
            B.qc_batch_set_chunk_pairs(batch, 3000)
            for m, (kt, ct, pt) in enumerate(ins):
                B.qc_batch_set_inputs(batch, m, kt, ct, pt, outs[m])
            B.qc_batch_eval(batch)
            sums = B.qc_batch_summaries(batch)
            for m, (e1, s1, _) in enumerate(singles):
                assert np.array_equal(outs[m].cpu().numpy().view(np.uint64), e1.view(np.uint64)), m
                assert sums[m]["e_re"] == s1["e_re"] and sums[m]["n_hits"] == s1["n_hits"]
        finally:
            B.qc_batch_destroy(batch)
    finally:
        for h in handles:
            B.qc_eloc_destroy(h)
