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


def allgather_combine(part: np.ndarray, dist, device=None) -> tuple[float, complex, float]:
    """Gather every rank's partials with torch.distributed (gloo on CPU tensors, NCCL on
    CUDA tensors) and combine them; every rank gets the same result."""
    import torch
    t = torch.as_tensor(np.asarray(part, dtype=np.float64), device=device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return combine(torch.stack(out).cpu().numpy())
