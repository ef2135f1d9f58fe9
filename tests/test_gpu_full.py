"""The accurate energy at scale (qc_eloc_export / qc_eloc_apply) against the oracle: the
exported connected set is every single and double excitation (the oracle's connected
union), in the documented order, with the Slater-Condon elements and diagonal of the
oracle; E_loc applied against psi on that set equals the oracle's FULL-mode E_loc."""
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


def _lookup(table_keys, table_psi, keys):
    """psi of each key from a sorted table (keys must all be present)."""
    tk = (table_keys[:, 1].astype(object) * (1 << 64) + table_keys[:, 0].astype(object))
    index = {int(k): i for i, k in enumerate(tk)}
    rows = np.array([index[(int(h) << 64) | int(l)] for l, h in keys], dtype=np.int64)
    return table_psi[rows]


def _run(B, ints, n_orb, n_elec, keys, counts, psi, table_keys, table_psi):
    import torch
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, n_orb, n_elec)
    try:
        P = B.qc_eloc_pairs_per_sample(h)
        kt = B.keys_to_tensor(keys)
        k, e, d = B.qc_eloc_export(h, kt)
        kx = k.cpu().numpy().view(np.uint64)
        pc = _lookup(table_keys, table_psi, kx)
        out = B.qc_eloc_apply(h, torch.from_numpy(psi).cuda(), torch.from_numpy(counts).cuda(), e, d,
                              torch.from_numpy(pc).cuda())
        summ = B.qc_eloc_summary_read(h)
        return P, kx, e.cpu().numpy(), d.cpu().numpy(), out.cpu().numpy(), summ
    finally:
        B.qc_eloc_destroy(h)


def test_export_apply_tiny_full_sector(B, orc):
    ints, s = I.make_workload("n14_e6_u1k")
    sector = orc.sector(14, 3, 3)
    psi_all = I.lognormal_psi(sector.shape[0], 1401)
    psi = _lookup(sector, psi_all, s.keys)
    P, kx, el, dg, eloc, summ = _run(B, ints, 14, 6, s.keys, s.counts, psi, sector, psi_all)
    assert P == 204 and kx.shape == (1000 * P, 2)
    want = orc.eloc(ints.h, ints.eri, 0.0, 14, s.keys, psi, sector, psi_all, mode=orc.FULL)
    err = np.abs(eloc - want) / np.maximum(1.0, np.abs(want))
    assert err.max() <= 1e-12
    m, var, w, n = orc.reduce(want, s.counts)
    assert abs(summ["energy"] - m) <= 1e-12 * abs(m) and summ["status"] == 0
    assert summ["n_pairs"] == 1000 * P and summ["n_hits"] == 0
    # the connected set: P distinct connected determinants per sample, union = the oracle's
    per = kx.reshape(1000, P, 2)
    even = np.uint64(0x5555555555555555)
    for r in range(0, 1000, 97):
        x = s.keys[r]
        seen = {(int(a), int(b)) for a, b in per[r]}
        assert len(seen) == P
        for a, b in per[r]:
            dx = bin(int(a) ^ int(x[0])).count("1") + bin(int(b) ^ int(x[1])).count("1")
            assert dx in (2, 4)
            assert bin(int(a) & int(even)).count("1") == bin(int(x[0]) & int(even)).count("1")
    union, _ = orc.dedup(kx)
    assert np.array_equal(union, orc.connected_union(14, s.keys))
    # the documented order: position 0 is alpha (occ[0] -> empty[0]); P - 1 the last alpha-beta
    x = s.keys[0]
    occa = [k for k in range(7) if (int(x[0]) >> (2 * k)) & 1]
    vira = [k for k in range(7) if not (int(x[0]) >> (2 * k)) & 1]
    first = int(x[0]) ^ (1 << (2 * occa[0])) ^ (1 << (2 * vira[0]))
    assert int(per[0, 0, 0]) == first
    # elements and diagonal against the Slater-Condon rules of the oracle
    rng = np.random.default_rng(5)
    for r, j in zip(rng.integers(0, 1000, 150), rng.integers(0, P, 150)):
        v, _ = orc.slater_condon(ints.h, ints.eri, 0.0, 14, s.keys[r], per[r, j])
        assert abs(el[r * P + j] - v) <= 1e-12 * max(1.0, abs(v))
    for r in range(0, 1000, 50):
        v, _ = orc.slater_condon(ints.h, ints.eri, 0.0, 14, s.keys[r], s.keys[r])
        assert abs(dg[r] - v) <= 1e-12 * max(1.0, abs(v))


def test_export_apply_n52(B, orc):
    K, n = 26, 60
    ints = I.make_integrals(K, 52, 5301)
    keys = I.rank_weighted_samples(K, 7, 7, n, seed=5302)
    counts = I.zipf_counts(n, 100 * n, 5303)
    table, _ = orc.dedup(np.concatenate([orc.connected_union(52, keys), keys]))
    tpsi = I.lognormal_psi(table.shape[0], 5304)
    psi = _lookup(table, tpsi, keys)
    P, kx, el, dg, eloc, summ = _run(B, ints, 52, 14, keys, counts, psi, table, tpsi)
    assert P == 25137
    want = orc.eloc(ints.h, ints.eri, 0.0, 52, keys, psi, table, tpsi, mode=orc.FULL)
    err = np.abs(eloc - want) / np.maximum(1.0, np.abs(want))
    assert err.max() <= 1e-10


def test_apply_invalid_and_zero_psi(B, orc):
    import torch
    ints, s = I.make_workload("n14_e6_u1k")
    keys = s.keys[:10].copy()
    keys[3, 0] ^= np.uint64(1)            # one electron more or less: not a determinant of the system
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 14, 6)
    try:
        k, e, d = B.qc_eloc_export(h, B.keys_to_tensor(keys))
        assert np.isnan(d.cpu().numpy()[3]) and np.isfinite(np.delete(d.cpu().numpy(), 3)).all()
        P = B.qc_eloc_pairs_per_sample(h)
        psi = s.psi[:10].copy()
        psi[6] = 0
        pc = torch.ones(10 * P, dtype=torch.complex128, device="cuda")
        out = B.qc_eloc_apply(h, torch.from_numpy(psi).cuda(), torch.from_numpy(s.counts[:10]).cuda(), e, d, pc)
        o = out.cpu().numpy()
        sm = B.qc_eloc_summary_read(h)
        assert np.isnan(o[3]) and np.isnan(o[6]) and sm["n_used"] == 8 and sm["status"] != 0
    finally:
        B.qc_eloc_destroy(h)
