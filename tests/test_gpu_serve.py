"""The serving form: requests submitted at any time, continuous batching on several
streams.  A request's result must be the same alone, in a mix of other molecules and cut
into row slices over many waves (bitwise, since batches run the single-molecule per-sample
code and the Eq. 1 reduction runs once over all rows), and equal to the handle API's; a
request that can never fit the memory budget is refused."""
import time

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


def _mol(n, ne, nu, seed):
    K = n // 2
    ints = I.make_integrals(K, n, seed)
    keys = I.rank_weighted_samples(K, ne // 2, ne // 2, nu, seed=seed + 1)
    return ints, keys, I.zipf_counts(nu, 40 * nu, seed + 2), I.lognormal_psi(nu, seed + 3)


def _wait(B, srv, t, limit_s=120.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        r = B.qc_eloc_poll(srv, t, 200_000)
        if r is not None:
            return r
    raise AssertionError("request did not finish")


def test_alone_equals_in_the_mix_and_handle_api(B, orc):
    import torch
    A = (28, 10, 1500, 1201)
    others = [(20, 8, 700, 1301), (40, 12, 900, 1401), (52, 14, 400, 1501), (24, 8, 2500, 1601)]
    mols = {key: _mol(n, ne, nu, sd) for key, (n, ne, nu, sd) in enumerate([A] + others, start=1)}
    srv = B.qc_server_create(0, 8 << 30, max_slots=16, n_streams=2)
    try:
        n, ne = A[0], A[1]
        ints, keys, counts, psi = mols[1]
        t = B.qc_eloc_submit(srv, ints.h, ints.eri, 0.0, n, ne, keys, counts, psi, mol_key=1)
        alone, e_alone = _wait(B, srv, t)
        assert alone["status"] == 0
        # the same request in a mix of four other molecules, submitted together
        tickets = {}
        for key, (nn, nee, nu, sd) in enumerate([A] + others, start=1):
            ints_k, keys_k, counts_k, psi_k = mols[key]
            tickets[key] = B.qc_eloc_submit(srv, ints_k.h, ints_k.eri, 0.0, nn, nee, keys_k, counts_k, psi_k,
                                            mol_key=key)
        res = {key: _wait(B, srv, tk) for key, tk in tickets.items()}
        assert np.array_equal(res[1][1].view(np.uint64), e_alone.view(np.uint64))
        assert res[1][0]["e_re"] == alone["e_re"]
        # each equals the handle API, and the oracle
        for key, (nn, nee, nu, sd) in enumerate([A] + others, start=1):
            ints_k, keys_k, counts_k, psi_k = mols[key]
            h = B.qc_eloc_create(ints_k.h, ints_k.eri, 0.0, nn, nee)
            try:
                e, _ = B.qc_eloc_eval(h, B.keys_to_tensor(keys_k), torch.from_numpy(counts_k).cuda(),
                                      torch.from_numpy(psi_k).cuda())
                assert np.array_equal(res[key][1].view(np.uint64), e.cpu().numpy().view(np.uint64)), key
            finally:
                B.qc_eloc_destroy(h)
            if key in (1, 3):
                want = orc.eloc(ints_k.h, ints_k.eri, 0.0, nn, keys_k, psi_k)
                err = np.abs(res[key][1] - want) / np.maximum(1.0, np.abs(want))
                assert err.max() <= 1e-6
        st = B.qc_server_stats(srv)
        assert st["in_flight"] == 0 and st["waiting"] == 0 and st["resident"] == 5
        for key in res:
            assert res[key][0]["t_submit"] <= res[key][0]["t_admit"] <= res[key][0]["t_start"] <= res[key][0]["t_done"]
    finally:
        B.qc_server_destroy(srv)


def test_wave_rows_cap_leaves_results_unchanged(B):
    """QC_SRV_OPT_WAVE_ROWS only decides which requests share a wave: with no cap, the default
    and a cap below every request's rows (each request alone, on the single-molecule path) the
    same requests give bitwise the same E_loc and energies; a negative cap is refused."""
    specs = [(28, 10, 1500, 2201), (20, 8, 700, 2301), (40, 12, 900, 2401), (24, 8, 2500, 2501)]
    mols = [_mol(n, ne, nu, sd) for n, ne, nu, sd in specs]
    runs = []
    for cap in (0, -1, 100):
        srv = B.qc_server_create(0, 8 << 30, max_slots=16, n_streams=2)
        try:
            if cap >= 0:
                B.qc_server_set_option(srv, B.QC_SRV_OPT_WAVE_ROWS, cap)
            tickets = [B.qc_eloc_submit(srv, ints.h, ints.eri, 0.0, n, ne, keys, counts, psi, mol_key=k + 1)
                       for k, ((n, ne, nu, sd), (ints, keys, counts, psi)) in enumerate(zip(specs, mols))]
            runs.append([_wait(B, srv, t) for t in tickets])
        finally:
            B.qc_server_destroy(srv)
    for k in range(len(specs)):
        for r in runs[1:]:
            assert r[k][0]["status"] == 0 and r[k][0]["e_re"] == runs[0][k][0]["e_re"]
            assert np.array_equal(r[k][1].view(np.uint64), runs[0][k][1].view(np.uint64)), k
    srv = B.qc_server_create(0, 1 << 30, max_slots=4, n_streams=1)
    try:
        with pytest.raises(B.QcError):
            B.qc_server_set_option(srv, B.QC_SRV_OPT_WAVE_ROWS, -5)
    finally:
        B.qc_server_destroy(srv)


def test_budget_refusal_and_eviction(B):
    ints, keys, counts, psi = _mol(24, 8, 500, 1701)
    srv = B.qc_server_create(0, 1 << 20, max_slots=4, n_streams=1)
    try:
        big = _mol(64, 16, 300, 1801)
        with pytest.raises(B.QcError) as ex:   # K^4 FP64 integrals alone exceed 1 MB
            B.qc_eloc_submit(srv, big[0].h, big[0].eri, 0.0, 64, 16, big[1], big[2], big[3])
        assert ex.value.status == -6
        # six molecules through a budget that holds about two: residents get evicted, all finish
        ts = [B.qc_eloc_submit(srv, ints.h, ints.eri, 0.1 * k, 24, 8, keys, counts, psi, mol_key=100 + k)
              for k in range(6)]
        outs = [_wait(B, srv, t) for t in ts]
        for k, (r, e) in enumerate(outs):
            assert r["status"] == 0
            assert np.allclose(e - outs[0][1], 0.1 * k, rtol=0, atol=1e-12)   # e_core shifts E_loc
    finally:
        B.qc_server_destroy(srv)


def test_sliced_requests_equal_whole(B):
    """With a small wave quantum every request runs as many row slices in many waves (and
    mixes with the others slice by slice); E_loc and the Eq. 1 energy stay bitwise those of
    one whole evaluation through the handle API."""
    import torch
    specs = [(40, 12, 3000, 2101), (52, 14, 2000, 2201), (28, 10, 1500, 2301)]
    mols = [_mol(*sp) for sp in specs]
    srv = B.qc_server_create(0, 8 << 30, max_slots=16, n_streams=2)
    try:
        with pytest.raises(B.QcError):
            B.qc_server_set_option(srv, B.QC_SRV_OPT_QUANTUM, -1)
        B.qc_server_set_option(srv, B.QC_SRV_OPT_QUANTUM, 2_000_000)   # a few hundred rows per wave
        tickets = [B.qc_eloc_submit(srv, m[0].h, m[0].eri, 0.0, sp[0], sp[1], m[1], m[2], m[3], mol_key=k + 1)
                   for k, (sp, m) in enumerate(zip(specs, mols))]
        res = [_wait(B, srv, t) for t in tickets]
        for sp, m, (r, e) in zip(specs, mols, res):
            assert r["status"] == 0
            h = B.qc_eloc_create(m[0].h, m[0].eri, 0.0, sp[0], sp[1])
            try:
                e1, _ = B.qc_eloc_eval(h, B.keys_to_tensor(m[1]), torch.from_numpy(m[2]).cuda(),
                                       torch.from_numpy(m[3]).cuda())
                s1 = B.qc_eloc_summary_read(h)
                assert np.array_equal(e.view(np.uint64), e1.cpu().numpy().view(np.uint64)), sp
                for f in ("e_re", "e_im", "var", "w", "n_hits", "n_pairs", "n_missing"):
                    assert r[f] == s1[f], (sp, f)
            finally:
                B.qc_eloc_destroy(h)
    finally:
        B.qc_server_destroy(srv)
