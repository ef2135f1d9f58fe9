"""A cost-weighted plan over two replicas (Alg. 2's split of the sample work, with costs
measured on the device), run one replica after the other on one GPU: each replica's pieces
(row ranges of molecules, evaluated against their whole sample tables) go through one batched
step, E_loc of every row is bitwise that of the unsplit batch, and the per-molecule energies
combined from the pieces' Eq. 1 partials equal the unsplit batch's and the oracle's."""
import numpy as np
import pytest

from paper_2506_23809_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (n_orb, n_elec, n_u): small enough for the oracle, uneven, one large enough for the join
MOLS = [(28, 10, 40000), (20, 6, 3000), (28, 10, 5000), (16, 6, 800), (32, 8, 2500), (24, 12, 1500)]


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
    out = []
    for i, (n, ne, nu) in enumerate(MOLS):
        K = n // 2
        ints = I.make_integrals(K, n, 8100 + i)
        keys = I.rank_weighted_samples(K, ne // 2, ne // 2, nu, seed=8200 + i)
        out.append((n, ne, ints, keys, I.zipf_counts(nu, 50 * nu, 8300 + i), I.lognormal_psi(nu, 8400 + i)))
    return out


def test_two_replica_plan_equals_unsplit(B, orc):
    import torch
    from paper_2506_23809_gb300 import shards
    mols = _molecules()
    handles = [B.qc_eloc_create(m[2].h, m[2].eri, 0.0, m[0], m[1]) for m in mols]
    try:
        dev = [(B.keys_to_tensor(m[3]), torch.from_numpy(m[4]).cuda(), torch.from_numpy(m[5]).cuda()) for m in mols]
        whole = [d + (torch.empty(len(m[3]), dtype=torch.complex128, device="cuda"),) for d, m in zip(dev, mols)]
        split = [d + (torch.empty(len(m[3]), dtype=torch.complex128, device="cuda"),) for d, m in zip(dev, mols)]
        # the unsplit batch
        batch = B.qc_batch_create(handles)
        for i, (k, c, p, e) in enumerate(whole):
            B.qc_batch_set_inputs(batch, i, k, c, p, e)
        B.qc_batch_eval(batch)
        ref = B.qc_batch_summaries(batch)
        B.qc_batch_destroy(batch)
        # the plan: costs measured on this device, two replicas
        costs = shards.calibrate_row_costs(B, handles, split)
        plan = shards.plan_pieces(costs, 2)
        assert all(len(p) > 0 for p in plan)
        assert sum(len(p) for p in plan) > len(mols)          # the largest molecule is cut
        for e in split:
            e[3].fill_(complex("nan"))
        parts = []
        for rep in plan:
            b, pp = shards.evaluate_pieces(B, handles, split, rep)
            B.qc_batch_destroy(b)
            parts += pp
        torch.cuda.synchronize()
        for (_, _, _, e0), (_, _, _, e1) in zip(whole, split):
            assert np.array_equal(e0.cpu().numpy().view(np.uint64), e1.cpu().numpy().view(np.uint64))
        got = shards.combine_pieces(len(mols), parts)
        for m, ((W, E, V), r) in enumerate(zip(got, ref)):
            assert W == r["w"]
            assert abs(E - r["energy"]) <= 1e-12 * abs(r["energy"]), m
            assert abs(V - r["var"]) <= 1e-9 * r["var"], m
            # and the oracle over all of the molecule's rows
            n, ne, ints, keys, counts, psi = mols[m]
            want = orc.eloc(ints.h, ints.eri, 0.0, n, keys, psi)
            mo, vo, wo, _ = orc.reduce(want, counts)
            assert W == wo and abs(E - mo) <= 1e-6 * abs(mo) and abs(V - vo) <= 1e-6 * vo
    finally:
        for h in handles:
            B.qc_eloc_destroy(h)


def test_set_rows_checks_its_range(B):
    import torch
    n, ne, ints, keys, counts, psi = _molecules()[3]
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, n, ne)
    try:
        batch = B.qc_batch_create([h])
        k, c, p = B.keys_to_tensor(keys), torch.from_numpy(counts).cuda(), torch.from_numpy(psi).cuda()
        e = torch.empty(len(keys), dtype=torch.complex128, device="cuda")
        B.qc_batch_set_inputs(batch, 0, k, c, p, e)
        for r0, r1 in ((-1, 5), (10, 5), (0, len(keys) + 1)):
            with pytest.raises(B.QcError):
                B.qc_batch_set_rows(batch, 0, r0, r1)
        with pytest.raises(B.QcError):
            B.qc_batch_set_rows(batch, 1, 0, 5)
        B.qc_batch_destroy(batch)
    finally:
        B.qc_eloc_destroy(h)
