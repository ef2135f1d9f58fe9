"""Checks of the seeded input generators (shapes, invariants, determinism) and of the
golden pair-count fixture against the closed form."""
import math
import os

import numpy as np

from paper_2506_23809_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_systems_pairs.txt")


def _popc(a):
    return np.array([bin(int(v)).count("1") for v in a])


def _spin_counts(keys, n_orb):
    ea = np.zeros(len(keys), dtype=np.int64)
    eb = np.zeros(len(keys), dtype=np.int64)
    for b in range(n_orb):
        bit = (keys[:, b >> 6] >> np.uint64(b & 63)) & np.uint64(1)
        if b % 2 == 0:
            ea += bit.astype(np.int64)
        else:
            eb += bit.astype(np.int64)
    return ea, eb


def _is_sorted_unique(keys):
    hi, lo = keys[:, 1], keys[:, 0]
    gt = (hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] > lo[:-1]))
    return bool(np.all(gt))


def test_tiny_workload():
    ints, s = I.make_workload("n14_e6_u1k")
    assert s.keys.shape == (1000, 2) and _is_sorted_unique(s.keys)
    ea, eb = _spin_counts(s.keys, 14)
    assert np.all(ea == 3) and np.all(eb == 3)
    assert s.counts.sum() == 100_000
    assert np.allclose(ints.h, ints.h.T)
    e = ints.eri
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)]:
        assert np.array_equal(e, e.transpose(perm))


def test_rank_weighted_generator_small():
    keys = I.rank_weighted_samples(10, 3, 3, 2000, seed=4)
    assert keys.shape == (2000, 2) and _is_sorted_unique(keys)
    ea, eb = _spin_counts(keys, 20)
    assert np.all(ea == 3) and np.all(eb == 3)
    ref = I.aufbau_key(10, 3, 3)
    assert any((k[0] == ref[0]) and (k[1] == ref[1]) for k in keys)
    again = I.rank_weighted_samples(10, 3, 3, 2000, seed=4)
    assert np.array_equal(keys, again)


def test_zipf_counts_exact_total():
    c = I.zipf_counts(10_000, 1_000_000, seed=3)
    assert c.sum() == 1_000_000 and c.min() >= 1


def test_golden_pairs_match_closed_form():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, n, ne, pairs = line.split()[:4]
        n, ne, pairs = int(n), int(ne), int(pairs)
        o = ne // 2
        v = n // 2 - o
        want = 2 * o * v + 2 * math.comb(o, 2) * math.comb(v, 2) + (o * v) ** 2
        assert pairs == want, name


def test_batched_and_serving_specs():
    specs = I.batched_molecule_specs()
    assert len(specs) == 64
    for s in specs:
        assert s["n_orb"] % 2 == 0 and 24 <= s["n_orb"] <= 120
        assert 2 <= s["n_elec"] <= s["n_orb"] // 2 and s["n_elec"] % 2 == 0
        assert 1 <= s["n_u"] <= 100_000
    reqs = I.serving_request_specs(50, 10.0)
    assert all(28 <= r["n_orb"] <= 128 for r in reqs)
    assert all(abs(r["n_elec"] - r["n_orb"] // 2) <= 4 for r in reqs)
    t = [r["t_arrive"] for r in reqs]
    assert t == sorted(t)
