"""Failure detection without faulting the GPU: a bounded device wait made to run out, a poll
that times out while its request is still running, and device allocations that fail on the
host.  Each ends in an error status the host reads, with the context still usable."""
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


def _tensors(B, s):
    import torch
    return B.keys_to_tensor(s.keys), torch.from_numpy(s.counts).cuda(), torch.from_numpy(s.psi).cuda()


@pytest.mark.parametrize("join", [1, 2])
def test_filter_wait_runs_out(B, orc, join):
    """QC_OPT_WAIT_LIMIT 0: every CTA's first wait for its filter copy gives up at once.  The
    CTA flags QC_FLAG_TIMEOUT, drains the copy with the full limit and leaves: the summary
    reports QC_ERR_TIMEOUT, no E_loc is written, and the next evaluation on the same handle
    (default limit) is correct."""
    import torch
    ints, s = I.make_workload("n14_e6_u1k")
    kt, ct, pt = _tensors(B, s)
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 14, 6)
    try:
        B.qc_eloc_set_option(h, B.QC_OPT_JOIN, join)
        B.qc_eloc_set_option(h, B.QC_OPT_WAIT_LIMIT, 0)
        out = torch.full((s.n_u,), complex(7.0, -7.0), dtype=torch.complex128, device="cuda")
        B.qc_eloc_eval(h, kt, ct, pt, eloc=out)
        sm = B.qc_eloc_summary_read(h)
        assert sm["status"] == -10 and sm["flags"] & 0x80
        got = out.cpu().numpy()
        assert np.all(got == complex(7.0, -7.0)), "a CTA that timed out wrote E_loc"
        assert sm["n_hits"] == 0
        B.qc_eloc_set_option(h, B.QC_OPT_WAIT_LIMIT, -1)
        e, _ = B.qc_eloc_eval(h, kt, ct, pt)
        sm = B.qc_eloc_summary_read(h)
        want = orc.eloc(ints.h, ints.eri, 0.0, 14, s.keys, s.psi)
        assert sm["status"] == 0
        assert np.abs(e.cpu().numpy() - want).max() <= 1e-6 * np.abs(want).max()
    finally:
        B.qc_eloc_destroy(h)


def test_poll_times_out_while_running(B):
    """qc_eloc_poll returns QC_PENDING (None here) when its timeout passes before the request
    is done, and the same ticket is returned complete by a later poll."""
    ints, s = I.make_workload("n76_e20_u200k")
    srv = B.qc_server_create(0, 16 << 30, max_slots=4, n_streams=1)
    try:
        t = B.qc_eloc_submit(srv, ints.h, ints.eri, 0.0, 76, 20, s.keys, s.counts, s.psi, precision=1, mol_key=76)
        assert B.qc_eloc_poll(srv, t, 0) is None
        assert B.qc_eloc_poll(srv, t, 500) is None          # 0.5 ms: the request takes tens of ms
        out = None
        for _ in range(600):
            out = B.qc_eloc_poll(srv, t, 100_000)
            if out is not None:
                break
        assert out is not None and out[0]["status"] == 0 and out[0]["n_used"] == s.n_u
    finally:
        B.qc_server_destroy(srv)


def test_allocation_failures_are_reported_and_leak_nothing(B, orc):
    """Every device allocation of handle creation and of the first evaluation (with the
    sample-space join) is made to fail in turn: each attempt returns QC_ERR_OOM, destroying
    the handle gives all memory back, and a clean evaluation afterwards is correct."""
    import torch
    K = 26
    ints = I.make_integrals(K, 52, 7101)
    keys = I.rank_weighted_samples(K, 7, 7, 20000, seed=7102)
    s = I.SampleSet(keys=keys, counts=I.zipf_counts(20000, 200000, 7103), psi=I.lognormal_psi(20000, 7104))
    kt, ct, pt = _tensors(B, s)
    out = torch.empty(s.n_u, dtype=torch.complex128, device="cuda")

    def attempt():
        h = None
        try:
            h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 52, 14)
            B.qc_eloc_eval(h, kt, ct, pt, eloc=out)
            return B.qc_eloc_summary_read(h)
        finally:
            if h is not None:
                B.qc_eloc_destroy(h)

    attempt()                        # loads every kernel this path launches
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for k in range(64):
            B.qc_test_fail_alloc(k)
            try:
                sm = attempt()
            except B.QcError as ex:
                assert ex.status == -5, ex
                failures += 1
                torch.cuda.synchronize()
                assert torch.cuda.mem_get_info()[0] == free0, f"allocation {k} failing leaked device memory"
                continue
            assert sm["status"] == 0
            break
    finally:
        B.qc_test_fail_alloc(-1)
    assert failures >= 10, failures      # handle tables, workspace, join index, ...
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    sm = attempt()
    rows = np.arange(0, s.n_u, 97)
    want = orc.eloc(ints.h, ints.eri, 0.0, 52, s.keys[rows], s.psi[rows], s.keys, s.psi)
    got = out.cpu().numpy()[rows]
    assert sm["status"] == 0 and np.abs(got - want).max() <= 1e-6 * max(1.0, np.abs(want).max())
