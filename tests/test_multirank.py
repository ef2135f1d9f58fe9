"""The N-rank path without a GPU: two gloo ranks each evaluate a block of rows against the
whole table (with the CPU oracle standing in for the device kernel) and combine their Eq. 1
partials with the exchange step of the package; the result equals the single-rank
reduction over all rows."""
import os
import socket

import numpy as np
import pytest

from paper_2506_23809_gb300 import shards


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2506_23809_gb300 import inputs as I
    ints, s = I.make_workload("n14_e6_u1k")
    lo, hi = shards.shard_rows(s.n_u, world, rank)
    el = oracle.eloc(ints.h, ints.eri, 0.0, 14, s.keys[lo:hi], s.psi[lo:hi], s.keys, s.psi, nthreads=1)
    m, var, w, n = oracle.reduce(el, s.counts[lo:hi])
    part = np.array([w, w * m.real, w * m.imag, w * var])
    W, E, V = shards.allgather_combine(part, dist)
    if rank == 0:
        np.save(out_path, np.array([W, E.real, E.imag, V]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_rows_cover_everything():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            blocks = [shards.shard_rows(n, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_combine_matches_pooled_moments():
    rng = np.random.default_rng(3)
    e = rng.normal(size=300) + 1j * rng.normal(size=300)
    c = rng.integers(1, 9, size=300).astype(float)
    W = c.sum()
    m = (c * e).sum() / W
    v = (c * np.abs(e - m) ** 2).sum() / W
    parts = []
    for lo, hi in ((0, 50), (50, 51), (51, 300)):
        w = c[lo:hi].sum()
        mr = (c[lo:hi] * e[lo:hi]).sum() / w
        vr = (c[lo:hi] * np.abs(e[lo:hi] - mr) ** 2).sum() / w
        parts.append([w, w * mr.real, w * mr.imag, w * vr])
    parts.append([0.0, 0.0, 0.0, 0.0])  # an empty shard
    W2, m2, v2 = shards.combine(parts)
    assert W2 == W and abs(m2 - m) < 1e-12 and abs(v2 - v) < 1e-12


def test_two_gloo_ranks_equal_one(tmp_path, orc):
    import multiprocessing as mp
    from paper_2506_23809_gb300 import inputs as I
    port = _free_port()
    out = str(tmp_path / "r0.npy")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    W, er, ei, V = np.load(out)
    ints, s = I.make_workload("n14_e6_u1k")
    el = orc.eloc(ints.h, ints.eri, 0.0, 14, s.keys, s.psi)
    m, var, w, n = orc.reduce(el, s.counts)
    assert W == w and abs(complex(er, ei) - m) <= 1e-12 * abs(m) and abs(V - var) <= 1e-10 * var


def test_plan_replicas_balances_and_covers():
    from paper_2506_23809_gb300 import inputs as I
    from paper_2506_23809_gb300.shards import job_cost, plan_replicas
    specs = I.batched_molecule_specs(64)

    def pairs(n_orb, ne):
        K, o = n_orb // 2, ne // 2
        v = K - o
        s = o * v
        return 2 * s + 2 * (o * (o - 1) // 2) * (v * (v - 1) // 2) + s * s
    jobs = [(sp["n_u"], pairs(sp["n_orb"], sp["n_elec"])) for sp in specs]
    for n_rep in (1, 2, 3, 8):
        plan = plan_replicas(jobs, n_rep)
        # every row of every job exactly once
        seen = {j: [] for j in range(len(jobs))}
        for rep in plan:
            for j, r0, r1 in rep:
                seen[j].append((r0, r1))
        for j, (n, _) in enumerate(jobs):
            rs = sorted(seen[j])
            assert rs[0][0] == 0 and rs[-1][1] == n and all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        loads = [sum(job_cost(r1 - r0, jobs[j][1]) for j, r0, r1 in rep) for rep in plan]
        total = sum(job_cost(n, p) for n, p in jobs)
        # within 10 % of a fair share (the largest molecule is cut into row ranges)
        assert max(loads) <= 1.10 * total / n_rep + 1e-9


def test_density_prediction():
    from paper_2506_23809_gb300.shards import density, predicted_unique
    d = density([50, 0, 30], [100, 0, 30])
    assert np.allclose(d, [0.5, 0.0, 1.0])
    assert np.allclose(predicted_unique([200, 10, 60], d), [100.0, 0.0, 60.0])


# ---------------------------------------------------------------------------------------
# a cost-weighted plan over two gloo ranks (the oracle stands in for the device kernel)
# ---------------------------------------------------------------------------------------
PLAN_MOLS = [(20, 6, 2400, 8601), (16, 6, 600, 8602), (24, 8, 900, 8603), (14, 6, 300, 8604)]


def _plan_inputs():
    from paper_2506_23809_gb300 import inputs as I
    mols = []
    for n, ne, nu, seed in PLAN_MOLS:
        K = n // 2
        ints = I.make_integrals(K, n, seed)
        keys = I.rank_weighted_samples(K, ne // 2, ne // 2, nu, seed=seed + 1)
        mols.append((n, ne, ints, keys, I.zipf_counts(nu, 20 * nu, seed + 2), I.lognormal_psi(nu, seed + 3)))
    return mols


def _plan(mols):
    """The plan every rank derives from the same costs (per-row costs from the oracle's hit
    counts and a fixed time per molecule: the inputs plan_pieces takes on the device)."""
    import oracle
    costs = []
    for n, ne, ints, keys, counts, psi in mols:
        _, det = oracle.eloc(ints.h, ints.eri, 0.0, n, keys, psi, details=True, nthreads=1)
        costs.append(shards.row_costs_from_timing(float(len(keys)), det["hits"]))
    return shards.plan_pieces(costs, 2)


def _plan_worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    mols = _plan_inputs()
    plan = _plan(mols)
    mine = []
    for m, r0, r1 in plan[rank]:
        n, ne, ints, keys, counts, psi = mols[m]
        el = oracle.eloc(ints.h, ints.eri, 0.0, n, keys[r0:r1], psi[r0:r1], keys, psi, nthreads=1)
        mo, var, w, _ = oracle.reduce(el, counts[r0:r1])
        mine.append((m, [w, w * mo.real, w * mo.imag, w * var]))
    got = [None] * world
    dist.all_gather_object(got, mine)
    res = shards.combine_pieces(len(mols), [x for g in got for x in g])
    if rank == 0:
        np.save(out_path, np.array([[W, E.real, E.imag, V] for W, E, V in res]))
    dist.barrier()
    dist.destroy_process_group()


def test_plan_pieces_cover_and_balance():
    rng = np.random.default_rng(5)
    costs = [rng.random(n) * s for n, s in ((5000, 5.0), (300, 1.0), (1200, 1.0), (40, 1.0), (1, 1.0))]
    total = sum(c.sum() for c in costs)
    for n_rep in (1, 2, 3, 8):
        plan = shards.plan_pieces(costs, n_rep)
        seen = {j: [] for j in range(len(costs))}
        for rep in plan:
            for j, r0, r1 in rep:
                seen[j].append((r0, r1))
        for j, c in enumerate(costs):
            rs = sorted(seen[j])
            assert rs[0][0] == 0 and rs[-1][1] == c.size and all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        loads = [sum(costs[j][r0:r1].sum() for j, r0, r1 in rep) for rep in plan]
        # a piece is at most about a fair share: no replica carries more than two shares
        assert max(loads) <= 2.0 * total / n_rep + 1e-9
        if n_rep == 2:
            assert max(loads) <= 1.10 * total / 2


def test_two_gloo_ranks_run_a_plan(tmp_path, orc):
    import multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "plan.npy")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_plan_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = np.load(out)
    mols = _plan_inputs()
    plan = _plan(mols)
    assert sum(len(p) for p in plan) > len(mols)          # a molecule is cut across the ranks
    for m, (n, ne, ints, keys, counts, psi) in enumerate(mols):
        el = orc.eloc(ints.h, ints.eri, 0.0, n, keys, psi)
        mo, var, w, _ = orc.reduce(el, counts)
        W, er, ei, V = got[m]
        assert W == w and abs(complex(er, ei) - mo) <= 1e-12 * abs(mo) and abs(V - var) <= 1e-10 * var


def _failing_worker(rank, world, port, out_dir, mode):
    """Rank 1 fails: 'status' -- its evaluation reports a nonzero status at the exchange;
    'dies' -- it raises before the exchange and exits.  Every surviving rank records what
    its exchange step raised, and how long it took."""
    import datetime
    import time

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    part = np.array([10.0 + rank, 1.0, 0.5, 2.0])
    if mode == "dies" and rank == 1:
        raise RuntimeError("rank 1 fails before the exchange")
    status = -10 if (mode == "status" and rank == 1) else 0   # QC_ERR_TIMEOUT
    t0 = time.time()
    try:
        shards.allgather_combine(part, dist, status=status)
        what = "combined"
    except shards.RankFailure as ex:
        what = "RankFailure " + " ".join(str(s) for s in ex.statuses)
    except RuntimeError as ex:  # the process group's error when a peer is gone
        what = "RuntimeError " + str(ex).splitlines()[0][:80]
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{what}\n{time.time() - t0:.3f}\n")


def _run_failing(tmp_path, mode):
    import multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, str(tmp_path), mode)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    out = {}
    for r in range(2):
        path = tmp_path / f"rank{r}.txt"
        if path.exists():
            what, dt = path.read_text().splitlines()
            out[r] = (what, float(dt))
    return codes, out


def test_a_failed_rank_status_reaches_every_rank(tmp_path):
    """A rank whose evaluation failed (here a bounded device wait that ran out) reports its
    status at the exchange step: every rank raises RankFailure naming it, and none combines
    partial sums that include the failed rank's."""
    codes, out = _run_failing(tmp_path, "status")
    assert codes == [0, 0]
    for r in range(2):
        assert out[r][0] == "RankFailure 0 -10", out[r]


def test_a_rank_that_dies_is_detected(tmp_path):
    """A rank that raises before the exchange step and exits: the surviving rank's collective
    ends with the process group's error (the peer closed its connection, or the 10 s
    timeout) rather than hanging, so it can stop before its next launch."""
    codes, out = _run_failing(tmp_path, "dies")
    assert codes[1] != 0 and 1 not in out
    assert codes[0] == 0 and out[0][0].startswith("RuntimeError"), out
    assert out[0][1] < 60.0
