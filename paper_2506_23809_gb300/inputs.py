"""Seeded synthetic inputs for the local-energy path (test and benchmark fixtures).

This module only *draws* inputs: one- and two-electron integrals, unique occupation
bitstrings, their counts and a wavefunction amplitude per bitstring.  It contains none
of the local-energy arithmetic (no excitation enumeration, no matrix elements, no
signs, no reductions), so both the CUDA path and the CPU oracle can be fed from it
without sharing any of the method.

Conventions (the occupation-number vector of Sec. II-A, interleaved spin orbitals):
  * spin orbital ``i`` <-> spatial orbital ``i >> 1``, spin alpha if ``i`` is even;
  * a bitstring is two little-endian uint64 words, bit ``i`` of word ``i >> 6``;
  * a sample table is sorted ascending as an unsigned 128-bit number whose high half
    is word 1.

The molecular integrals the paper uses (N2, PH3, LiCl, Fe2S2, H50, C6H6; Sec. IV) are
not available here; the generators below produce seeded stand-ins with the same shapes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Integrals", "SampleSet", "make_integrals", "aufbau_key", "pack_occupations",
    "sort_keys", "sector_keys", "uniform_samples", "rank_weighted_samples",
    "multinomial_counts", "zipf_counts", "lognormal_psi", "WORKLOADS", "make_workload",
    "batched_molecule_specs", "serving_request_specs", "PAPER_SYSTEMS", "paper_system_workload",
]


@dataclass
class Integrals:
    """Spatial-orbital integrals: ``h[p, q]`` and chemist-notation ``eri[p, q, r, s] = (pq|rs)``."""
    h: np.ndarray
    eri: np.ndarray
    e_core: float = 0.0

    @property
    def n_spatial(self) -> int:
        return self.h.shape[0]


@dataclass
class SampleSet:
    """Unique sorted bitstrings with counts and complex amplitudes (row-aligned)."""
    keys: np.ndarray          # uint64 [n_u, 2]
    counts: np.ndarray        # int64  [n_u]
    psi: np.ndarray           # complex128 [n_u]
    meta: dict = field(default_factory=dict)

    @property
    def n_u(self) -> int:
        return self.keys.shape[0]


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------------
# integrals
# ----------------------------------------------------------------------------------
def make_integrals(n_spatial: int, rank: int, seed: int, e_core: float = 0.0) -> Integrals:
    """h: symmetric, diagonal -U(1,5), off-diagonal N(0, 0.1 exp(-|p-q|/2)).

    (pq|rs) = sum_k L^k_pq L^k_rs with L^k symmetric K x K, entries N(0, 0.3): this has
    the full 8-fold permutational symmetry of real orbitals by construction.
    """
    rng = _rng(seed)
    K = n_spatial
    h = np.zeros((K, K))
    idx = np.arange(K)
    dist = np.abs(idx[:, None] - idx[None, :])
    off = rng.normal(0.0, 1.0, size=(K, K)) * (0.1 * np.exp(-dist / 2.0))
    off = np.triu(off, 1)
    h = off + off.T
    h[idx, idx] = -rng.uniform(1.0, 5.0, size=K)
    L = rng.normal(0.0, 0.3, size=(rank, K, K))
    iu, ju = np.triu_indices(K)
    Lp = L[:, iu, ju]                        # [rank, npair] factor over unordered pairs
    V = Lp.T @ Lp                            # (pq|rs) over pairs p<=q, r<=s
    V = 0.5 * (V + V.T)                      # exactly symmetric under (pq) <-> (rs)
    pair = np.zeros((K, K), dtype=np.int64)
    pair[iu, ju] = np.arange(len(iu))
    pair[ju, iu] = np.arange(len(iu))
    eri = V[pair[:, :, None, None], pair[None, None, :, :]]
    return Integrals(h=np.ascontiguousarray(h), eri=np.ascontiguousarray(eri), e_core=float(e_core))


# ----------------------------------------------------------------------------------
# bitstrings
# ----------------------------------------------------------------------------------
def pack_occupations(occ_alpha: np.ndarray, occ_beta: np.ndarray) -> np.ndarray:
    """Boolean spatial occupations [M, K] per spin -> uint64 [M, 2] interleaved keys."""
    occ_alpha = np.asarray(occ_alpha, dtype=bool)
    occ_beta = np.asarray(occ_beta, dtype=bool)
    M, K = occ_alpha.shape
    bits = np.zeros((M, 128), dtype=bool)
    bits[:, 0:2 * K:2] = occ_alpha
    bits[:, 1:2 * K:2] = occ_beta
    weights = (np.uint64(1) << np.arange(64, dtype=np.uint64))
    lo = (bits[:, :64].astype(np.uint64) * weights).sum(axis=1, dtype=np.uint64)
    hi = (bits[:, 64:].astype(np.uint64) * weights).sum(axis=1, dtype=np.uint64)
    return np.stack([lo, hi], axis=1)


def sort_keys(keys: np.ndarray) -> np.ndarray:
    """Permutation sorting uint64[M,2] keys ascending as unsigned 128-bit (hi = word 1)."""
    return np.lexsort((keys[:, 0], keys[:, 1]))


def aufbau_key(n_spatial: int, n_alpha: int, n_beta: int) -> np.ndarray:
    oa = np.zeros((1, n_spatial), dtype=bool)
    ob = np.zeros((1, n_spatial), dtype=bool)
    oa[0, :n_alpha] = True
    ob[0, :n_beta] = True
    return pack_occupations(oa, ob)[0]


def _spin_strings(K: int, n: int) -> np.ndarray:
    """All boolean occupation rows with n of K orbitals occupied."""
    import itertools
    rows = np.zeros((math.comb(K, n), K), dtype=bool)
    for r, c in enumerate(itertools.combinations(range(K), n)):
        rows[r, list(c)] = True
    return rows


def sector_keys(n_spatial: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Every bitstring of the (n_alpha, n_beta) sector, sorted (small K only)."""
    A = _spin_strings(n_spatial, n_alpha)
    B = _spin_strings(n_spatial, n_beta)
    oa = np.repeat(A, len(B), axis=0)
    ob = np.tile(B, (len(A), 1))
    keys = pack_occupations(oa, ob)
    return np.ascontiguousarray(keys[sort_keys(keys)])


def uniform_samples(n_spatial: int, n_alpha: int, n_beta: int, n_u: int, seed: int) -> np.ndarray:
    """n_u distinct sector bitstrings drawn uniformly without replacement, sorted."""
    rng = _rng(seed)
    allk = sector_keys(n_spatial, n_alpha, n_beta)
    if n_u > len(allk):
        raise ValueError("n_u exceeds the sector dimension")
    pick = rng.choice(len(allk), size=n_u, replace=False)
    keys = allk[np.sort(pick)]
    return np.ascontiguousarray(keys)


def _random_subset_mask(rng, M: int, n: int, k: np.ndarray) -> np.ndarray:
    """Row-wise uniformly random subsets of size k[m] out of n positions: the k[m]
    smallest of n i.i.d. uniforms in each row."""
    if n == 0:
        return np.zeros((M, 0), dtype=bool)
    r = rng.random((M, n))
    srt = np.sort(r, axis=1)
    thr = np.where(k > 0, srt[np.arange(M), np.maximum(k, 1) - 1], -1.0)
    return r <= thr[:, None]


def rank_weighted_samples(n_spatial: int, n_alpha: int, n_beta: int, n_u: int, seed: int,
                          decay: float = 0.3, batch: int = 1 << 18) -> np.ndarray:
    """Distinct bitstrings drawn from a Boltzmann-like law over excitation rank.

    Rank k (relative to the Aufbau determinant, alpha plus beta excitations) has weight
    proportional to decay**k; within a rank the split (k_a, k_b) is weighted by the number
    of determinants of that split and the determinant is uniform within the split.
    Duplicates are rejected; the first n_u distinct draws are kept, then sorted.
    """
    rng = _rng(seed)
    K = n_spatial
    oa, va, ob, vb = n_alpha, K - n_alpha, n_beta, K - n_beta
    kamax, kbmax = min(oa, va), min(ob, vb)
    splits = []
    for ka in range(kamax + 1):
        for kb in range(kbmax + 1):
            n_det = math.comb(oa, ka) * math.comb(va, ka) * math.comb(ob, kb) * math.comb(vb, kb)
            splits.append((ka, kb, n_det))
    kmax = kamax + kbmax
    rank_w = np.array([decay ** k for k in range(kmax + 1)])
    rank_w /= rank_w.sum()
    per_rank = {k: [(ka, kb, nd) for (ka, kb, nd) in splits if ka + kb == k] for k in range(kmax + 1)}
    total_dets = sum(nd for (_, _, nd) in splits)
    if n_u > total_dets:
        raise ValueError("n_u exceeds the sector dimension")
    # keep the first n_u distinct draws: dedupe every batch against the distinct keys so
    # far, remembering each key's first draw index
    aufbau = aufbau_key(K, n_alpha, n_beta)
    u_lo = np.empty(0, dtype=np.uint64)
    u_hi = np.empty(0, dtype=np.uint64)
    first = np.empty(0, dtype=np.int64)
    drawn = 0
    while len(first) < n_u:
        ranks = rng.choice(kmax + 1, size=batch, p=rank_w)
        ka = np.empty(batch, dtype=np.int64)
        kb = np.empty(batch, dtype=np.int64)
        for k in range(kmax + 1):
            sel = np.nonzero(ranks == k)[0]
            if sel.size == 0:
                continue
            opts = per_rank[k]
            w = np.array([nd for (_, _, nd) in opts], dtype=float)
            w /= w.sum()
            pick = rng.choice(len(opts), size=sel.size, p=w)
            ka[sel] = np.array([o[0] for o in opts])[pick]
            kb[sel] = np.array([o[1] for o in opts])[pick]
        keys = np.empty((batch, 2), dtype=np.uint64)
        keys[:] = aufbau
        ex = np.nonzero(ranks > 0)[0]          # rank 0 is the Aufbau determinant itself
        m = ex.size
        if m:
            holes_a = _random_subset_mask(rng, m, oa, ka[ex])
            parts_a = _random_subset_mask(rng, m, va, ka[ex])
            holes_b = _random_subset_mask(rng, m, ob, kb[ex])
            parts_b = _random_subset_mask(rng, m, vb, kb[ex])
            occ_a = np.concatenate([~holes_a, parts_a], axis=1)
            occ_b = np.concatenate([~holes_b, parts_b], axis=1)
            keys[ex] = pack_occupations(occ_a, occ_b)
        lo = np.concatenate([u_lo, keys[:, 0]])
        hi = np.concatenate([u_hi, keys[:, 1]])
        fi = np.concatenate([first, drawn + np.arange(batch, dtype=np.int64)])
        order = np.lexsort((fi, lo, hi))
        lo, hi, fi = lo[order], hi[order], fi[order]
        keep = np.ones(len(lo), dtype=bool)
        keep[1:] = (lo[1:] != lo[:-1]) | (hi[1:] != hi[:-1])
        u_lo, u_hi, first = lo[keep], hi[keep], fi[keep]
        drawn += batch
    sel = np.argsort(first, kind="stable")[:n_u]
    keys = np.stack([u_lo[sel], u_hi[sel]], axis=1)
    return np.ascontiguousarray(keys[sort_keys(keys)])


# ----------------------------------------------------------------------------------
# counts and amplitudes
# ----------------------------------------------------------------------------------
def multinomial_counts(n_u: int, total: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    return rng.multinomial(total, np.full(n_u, 1.0 / n_u)).astype(np.int64)


def zipf_counts(n_u: int, total: int, seed: int, s: float = 1.2) -> np.ndarray:
    """Zipf(s) weights over a random permutation, each count >= 1, summing to ``total``
    exactly (largest-remainder rounding of the part above the floor of one)."""
    if total < n_u:
        raise ValueError("total must be >= n_u")
    rng = _rng(seed)
    perm = rng.permutation(n_u)
    w = 1.0 / np.power(np.arange(1, n_u + 1, dtype=float), s)
    w = w[np.argsort(perm)]  # rank perm[i] -> sample i
    extra = total - n_u
    share = w / w.sum() * extra
    base = np.floor(share).astype(np.int64)
    rem = extra - int(base.sum())
    if rem > 0:
        frac = share - base
        top = np.argsort(-frac, kind="stable")[:rem]
        base[top] += 1
    return (base + 1).astype(np.int64)


def lognormal_psi(n_u: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """log|psi| ~ N(0, sigma), phase ~ U(0, 2 pi)."""
    rng = _rng(seed)
    la = rng.normal(0.0, sigma, size=n_u)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_u)
    return np.exp(la) * (np.cos(ph) + 1j * np.sin(ph))


# ----------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------
WORKLOADS = {
    # tiny: N=14 spin orbitals, 6 electrons, 1,000 uniform samples of the 1,225-dim sector
    "n14_e6_u1k": dict(n_orb=14, n_elec=6, rank=14, n_u=1000, sampler="uniform",
                       counts=("multinomial", 100_000), seed=1401),
    # plain FP64 GPU workload: N=52, 14 electrons, 1e5 rank-weighted samples, Zipf counts
    "n52_e14_u100k": dict(n_orb=52, n_elec=14, rank=52, n_u=100_000, sampler="rank",
                          counts=("zipf", 10_000_000), seed=5201),
    # precision form: N=76, 20 electrons, 2e5 samples (FP32 integrals on the device)
    "n76_e20_u200k": dict(n_orb=76, n_elec=20, rank=76, n_u=200_000, sampler="rank",
                          counts=("zipf", 20_000_000), seed=7601),
}


# The paper's molecular shapes (spin orbitals, electrons): N2, PH3 and LiCl of Table I; Fe2S2,
# H50 and C6H6 of Sec. IV-B (C6H6's electron count is not given: half filling).  Their
# integrals are not available; each gets seeded synthetic integrals of its size (rank N), and
# up to 1e5 rank-weighted unique samples -- at most half of a small sector.
PAPER_SYSTEMS = [("N2", 20, 14), ("PH3", 24, 18), ("LiCl", 28, 20), ("Fe2S2", 40, 30), ("H50", 100, 50),
                 ("C6H6", 120, 60)]


def paper_system_workload(name: str, n_u_max: int = 100_000):
    """(spec dict, Integrals, SampleSet) of one paper-shaped system: Zipf counts summing to
    100 per sample, lognormal complex psi."""
    n_orb, n_elec = {n: (a, b) for n, a, b in PAPER_SYSTEMS}[name]
    K, o = n_orb // 2, n_elec // 2
    n_u = min(n_u_max, math.comb(K, o) ** 2 // 2)
    seed = 9000 + n_orb
    ints = make_integrals(K, n_orb, seed)
    keys = rank_weighted_samples(K, o, o, n_u, seed=seed + 1)
    s = SampleSet(keys=keys, counts=zipf_counts(n_u, 100 * n_u, seed + 2), psi=lognormal_psi(n_u, seed + 3),
                  meta=dict(name=name))
    return dict(name=name, n_orb=n_orb, n_elec=n_elec, n_u=n_u, seed=seed), ints, s


def make_workload(name: str = None, *, n_orb: int = None, n_elec: int = None, rank: int = None,
                  n_u: int = None, sampler: str = "rank", counts=("zipf", None), seed: int = 0):
    """Returns (Integrals, SampleSet) for a named workload or explicit parameters."""
    if name is not None:
        spec = dict(WORKLOADS[name])
        n_orb, n_elec, rank, n_u = spec["n_orb"], spec["n_elec"], spec["rank"], spec["n_u"]
        sampler, counts, seed = spec["sampler"], spec["counts"], spec["seed"]
    if rank is None:
        rank = n_orb
    K = n_orb // 2
    na = nb = n_elec // 2
    ints = make_integrals(K, rank, seed)
    if sampler == "uniform":
        keys = uniform_samples(K, na, nb, n_u, seed + 1)
    elif sampler == "rank":
        keys = rank_weighted_samples(K, na, nb, n_u, seed + 1)
    else:
        raise ValueError(sampler)
    kind, total = counts
    if total is None:
        total = 100 * n_u
    if kind == "multinomial":
        c = multinomial_counts(n_u, total, seed + 2)
    else:
        c = zipf_counts(n_u, total, seed + 2)
    psi = lognormal_psi(n_u, seed + 3)
    meta = dict(name=name, n_orb=n_orb, n_elec=n_elec, rank=rank, n_u=n_u, sampler=sampler,
                counts=kind, total=int(total), seed=seed)
    return ints, SampleSet(keys=keys, counts=c, psi=psi, meta=meta)


def batched_molecule_specs(n_mol: int = 64, seed: int = 6400):
    """Per-molecule (n_orb, n_elec, n_u, seed) for the many-molecule batched form:
    N even uniform in 24..120, n_elec = N/2 - 2*U{0..N/4}, rounded down to even (S_z = 0)
    and clamped to >= 2,
    n_u log-uniform in [1e3, 1e5] (at most a quarter of a small sector)."""
    rng = _rng(seed)
    specs = []
    for m in range(n_mol):
        N = int(rng.integers(12, 61)) * 2
        ne = N // 2 - 2 * int(rng.integers(0, N // 4 + 1))
        ne -= ne % 2          # S_z = 0 needs an even count: round an odd N/2 down
        ne = max(ne, 2)
        n_u = int(round(10 ** rng.uniform(3.0, 5.0)))
        n_u = min(n_u, math.comb(N // 2, ne // 2) ** 2 // 4)  # small sectors: a quarter at most
        specs.append(dict(n_orb=N, n_elec=ne, n_u=n_u, seed=seed + 17 * (m + 1)))
    return specs


def serving_request_specs(n_req: int, rate_hz: float, seed: int = 9100,
                          nu_median: float = 3e4, nu_clip=(1_000, 1_000_000)):
    """Poisson arrivals; N even uniform in 28..128; n_elec uniform over the even counts
    within 4 of half filling (S_z = 0);
    n_u lognormal (median nu_median) clipped to nu_clip."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for r in range(n_req):
        t += rng.exponential(1.0 / rate_hz)
        N = int(rng.integers(14, 65)) * 2
        half = N // 2
        choices = [e for e in range(half - 4, half + 5) if e % 2 == 0 and 2 <= e <= N - 2]
        ne = choices[int(rng.integers(0, len(choices)))]
        n_u = int(np.clip(round(nu_median * math.exp(rng.normal(0.0, 1.0))), *nu_clip))
        out.append(dict(t_arrive=t, n_orb=N, n_elec=ne, n_u=n_u, seed=seed + 31 * (r + 1)))
    return out
