"""Sample sharding across ranks and the one exchange step of the path.

Alg. 3 partitions the unique samples across processes and ends with an all-reduce of the
energy sums; Eq. 1 is the count-weighted mean.  Here each rank evaluates a contiguous block
of rows against the whole table; its summary gives the partials (W_r, sum c E over its rows,
W_r * var_r).  Gathering these 4 doubles per rank and combining them (Chan, Golub and
LeVeque's pairwise update of mean and second moment) yields the global mean and variance.
"""
from __future__ import annotations

import numpy as np


def shard_rows(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [lo, hi) block of rows for `rank`; the first n_total % world ranks get one more."""
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def partials(summary: dict) -> np.ndarray:
    """(W, Re sum cE, Im sum cE, W * var) of one shard from a qc_eloc summary."""
    w = float(summary["w"])
    return np.array([w, summary["sum_ce_re"], summary["sum_ce_im"], w * summary["var"]], dtype=np.float64)


def combine(parts) -> tuple[float, complex, float]:
    """Global (W, Ebar, var) from stacked shard partials [[W, Sre, Sim, W var], ...]."""
    p = np.asarray(parts, dtype=np.float64).reshape(-1, 4)
    keep = p[:, 0] > 0
    p = p[keep]
    W = p[:, 0].sum()
    if W == 0:
        return 0.0, complex(np.nan, np.nan), float("nan")
    ebar = complex(p[:, 1].sum(), p[:, 2].sum()) / W
    means = (p[:, 1] + 1j * p[:, 2]) / p[:, 0]
    var = (p[:, 3].sum() + (p[:, 0] * np.abs(means - ebar) ** 2).sum()) / W
    return float(W), ebar, float(var)


class RankFailure(RuntimeError):
    """A rank reported a failed evaluation (a nonzero qc_eloc status) at the exchange step."""

    def __init__(self, statuses):
        bad = {r: s for r, s in enumerate(statuses) if s != 0}
        super().__init__(f"ranks reported failed evaluations (rank: status): {bad}")
        self.statuses = list(statuses)


def allgather_combine(part: np.ndarray, dist, device=None, status: int = 0) -> tuple[float, complex, float]:
    """Gather every rank's partials with torch.distributed (gloo on CPU tensors, NCCL on
    CUDA tensors) and combine them; every rank gets the same result.  Each rank also sends
    the status of its evaluation: if any rank's is nonzero, every rank raises RankFailure
    instead of combining (a rank whose kernel ran out of a bounded wait, say, must not
    contribute its partial sums).  A rank that never reaches the exchange (it died) ends the
    others' collective with the process group's error or timeout."""
    import torch
    v = np.append(np.asarray(part, dtype=np.float64).reshape(4), float(status))
    t = torch.as_tensor(v, device=device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    g = torch.stack(out).cpu().numpy()
    statuses = [int(s) for s in g[:, 4]]
    if any(s != 0 for s in statuses):
        raise RankFailure(statuses)
    return combine(g[:, :4])


# ---------------------------------------------------------------------------------------
# Cost-weighted plans across replicas (many molecules, uneven sizes): Alg. 2 balances the
# unique samples of partitions by predicted counts; here molecules are cut by measured cost
# ---------------------------------------------------------------------------------------
def job_cost(n_rows: int, pairs_per_sample: int, per_sample: float = 4096.0) -> float:
    """Estimated work of n_rows samples of one molecule: every sample enumerates the same
    number of connected pairs, plus a per-sample set-up share (in pair equivalents)."""
    return float(n_rows) * (float(pairs_per_sample) + per_sample)


def plan_replicas(jobs, n_replicas: int, per_sample: float = 4096.0, min_rows: int = 1):
    """Split jobs [(n_rows, pairs_per_sample), ...] over replicas so that the estimated
    work of each is about equal.  Whole jobs go longest first to the least-loaded replica;
    a job larger than a fair share is cut into row ranges first, so no replica waits on one
    long molecule.  Returns, per replica, a list of (job index, row0, row1)."""
    if n_replicas < 1:
        raise ValueError("n_replicas >= 1")
    costs = [job_cost(n, p, per_sample) for n, p in jobs]
    total = sum(costs)
    share = total / n_replicas if total > 0 else 0.0
    pieces = []           # (cost, job, r0, r1)
    for j, ((n, p), c) in enumerate(zip(jobs, costs)):
        if n <= 0:
            continue
        if share > 0 and c > share and n > min_rows:
            k = min(n, max(2, int(np.ceil(c / share))))
            for q in range(k):
                r0, r1 = (n * q) // k, (n * (q + 1)) // k
                if r1 > r0:
                    pieces.append((job_cost(r1 - r0, p, per_sample), j, r0, r1))
        else:
            pieces.append((c, j, 0, n))
    pieces.sort(key=lambda t: (-t[0], t[1], t[2]))
    load = [0.0] * n_replicas
    plan = [[] for _ in range(n_replicas)]
    for c, j, r0, r1 in pieces:
        r = min(range(n_replicas), key=lambda i: (load[i], i))
        load[r] += c
        plan[r].append((j, r0, r1))
    for p in plan:
        p.sort()
    return plan


def row_costs_from_timing(ms: float, hits) -> np.ndarray:
    """Per-row cost (ms) of one molecule from a measured evaluation: its device time `ms`
    spread over the rows in proportion to (mean hits + the row's hits) -- every row pays its
    set-up and scans, and the rows near the reference determinant find many more hits."""
    h = np.asarray(hits, dtype=np.float64)
    if h.size == 0:
        return h
    w = h.mean() + h + 1e-9
    return float(ms) * w / w.sum()


def plan_pieces(row_costs, n_replicas: int):
    """Cost-weighted plan over replicas (Alg. 2's split, with costs instead of sample counts):
    row_costs is one array of per-row costs per molecule.  A molecule whose cost exceeds a
    fair share (total / n_replicas) is cut into contiguous row ranges of about equal cost;
    pieces then go longest first to the least-loaded replica.  Returns, per replica, a sorted
    list of (molecule, row0, row1); every row of every molecule is in exactly one piece."""
    if n_replicas < 1:
        raise ValueError("n_replicas >= 1")
    costs = [np.asarray(c, dtype=np.float64) for c in row_costs]
    totals = [float(c.sum()) for c in costs]
    share = sum(totals) / n_replicas if sum(totals) > 0 else 0.0
    pieces = []           # (cost, molecule, r0, r1)
    for j, (c, tot) in enumerate(zip(costs, totals)):
        n = c.size
        if n == 0:
            continue
        if share > 0 and tot > share and n > 1:
            k = min(n, int(np.ceil(tot / share)))
            cum = np.cumsum(c)
            cuts = [0] + [int(np.searchsorted(cum, tot * q / k, side="left")) + 1 for q in range(1, k)] + [n]
            cuts = sorted(set(min(max(x, 0), n) for x in cuts))
            for r0, r1 in zip(cuts, cuts[1:]):
                if r1 > r0:
                    pieces.append((float(c[r0:r1].sum()), j, r0, r1))
        else:
            pieces.append((tot, j, 0, n))
    pieces.sort(key=lambda t: (-t[0], t[1], t[2]))
    load = [0.0] * n_replicas
    plan = [[] for _ in range(n_replicas)]
    for c, j, r0, r1 in pieces:
        r = min(range(n_replicas), key=lambda i: (load[i], i))
        load[r] += c
        plan[r].append((j, r0, r1))
    for p in plan:
        p.sort()
    return plan


def combine_pieces(n_mol: int, pieces):
    """Per-molecule (W, Ebar, var) from the partials of its pieces: pieces is a list of
    (molecule, partials) with partials as returned by ``partials``."""
    per = [[] for _ in range(n_mol)]
    for m, part in pieces:
        per[m].append(part)
    return [combine(p) if p else (0.0, complex(np.nan, np.nan), float("nan")) for p in per]


def calibrate_row_costs(binding, handles, inputs, stream=None):
    """Per-row costs of every molecule for plan_pieces, from one timed evaluation each on this
    device: its main-kernel time spread over its rows by their hit counts."""
    import torch
    out = []
    for h, (keys, counts, psi, eloc) in zip(handles, inputs):
        binding.qc_eloc_set_option(h, binding.QC_OPT_TIMING, 1)
        _, d = binding.qc_eloc_eval(h, keys, counts, psi, eloc=eloc, diagnostics=True, stream=stream)
        ms = binding.qc_eloc_timings(h)[1]
        out.append(row_costs_from_timing(ms, d["hit_count"].to(torch.int64).cpu().numpy()))
    return out


def evaluate_pieces(binding, handles, inputs, pieces, stream=None, autotune=False, graph=False):
    """One replica's share of a plan as one batched step: a batch entry per piece (its
    molecule's handle and whole sample set; only the piece's rows are evaluated and reduced).
    inputs[m] = (keys, counts, psi, eloc) device tensors of molecule m; E_loc of the piece's
    rows lands in eloc.  Returns (the batch, [(molecule, partials)] per piece); the caller
    destroys the batch."""
    batch = binding.qc_batch_create([handles[m] for m, _, _ in pieces])
    for i, (m, r0, r1) in enumerate(pieces):
        keys, counts, psi, eloc = inputs[m]
        binding.qc_batch_set_inputs(batch, i, keys, counts, psi, eloc)
        binding.qc_batch_set_rows(batch, i, r0, r1)
    if autotune:
        binding.qc_batch_autotune(batch, stream, iters=2)
    if graph:
        binding.qc_batch_graph_launch(batch, stream)
    else:
        binding.qc_batch_eval(batch, stream)
    sums = binding.qc_batch_summaries(batch, stream)
    return batch, [(m, partials(sm)) for (m, _, _), sm in zip(pieces, sums)]


def predicted_unique(sample_counts, density_prev) -> np.ndarray:
    """The density-aware estimate of Alg. 2: the unique samples a partition will hold is its
    sample count times the unique-to-sample ratio d = unique / counts measured for it in the
    previous iteration (the sample distribution changes slowly between iterations)."""
    return np.asarray(sample_counts, dtype=np.float64) * np.asarray(density_prev, dtype=np.float64)


def density(n_unique, n_counts) -> np.ndarray:
    """Alg. 2's density metric d = unique / counts (0 where nothing was drawn)."""
    u = np.asarray(n_unique, dtype=np.float64)
    c = np.asarray(n_counts, dtype=np.float64)
    return np.divide(u, c, out=np.zeros_like(u), where=c > 0)
