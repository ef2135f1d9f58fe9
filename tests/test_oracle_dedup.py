"""Pins for the oracle's sample-table construction (dedup): against brute force with Python
integers (a set and a counter), and against the invariants of the table (strictly
increasing 128-bit keys, counts summing to the stream length)."""
import collections

import numpy as np
import pytest

import oracle
from paper_2506_23809_gb300 import inputs as I


def _brute(raw):
    c = collections.Counter((int(r[1]) << 64) | int(r[0]) for r in raw)
    keys = sorted(c)
    out = np.array([[k & ((1 << 64) - 1), k >> 64] for k in keys], dtype=np.uint64).reshape(-1, 2)
    return out, np.array([c[k] for k in keys], dtype=np.int64)


@pytest.mark.parametrize("n,n_bits,seed", [(1, 8, 1), (500, 6, 2), (3000, 70, 3), (2000, 128, 4)])
def test_dedup_equals_brute_force(n, n_bits, seed):
    import random
    rnd = random.Random(seed)
    pool = [rnd.getrandbits(n_bits) for _ in range(max(1, n // 3))]   # repeats are common
    vals = [rnd.choice(pool) for _ in range(n)]
    raw = np.array([[v & ((1 << 64) - 1), v >> 64] for v in vals], dtype=np.uint64)
    keys, counts = oracle.dedup(raw)
    bk, bc = _brute(raw)
    assert np.array_equal(keys, bk) and np.array_equal(counts, bc)


def test_dedup_of_expanded_sample_set_is_the_set():
    """The bench stream: a unique sorted sample set expanded by its counts and shuffled
    dedups back to exactly that set and those counts; the table is strictly increasing."""
    s = I.make_workload("n14_e6_u1k")[1]
    rng = np.random.default_rng(7)
    raw = np.repeat(s.keys, s.counts, axis=0)
    raw = raw[rng.permutation(raw.shape[0])]
    keys, counts = oracle.dedup(raw)
    assert np.array_equal(keys, s.keys) and np.array_equal(counts, s.counts)
    hi, lo = keys[:, 1].astype(object), keys[:, 0].astype(object)
    k = [(int(a) << 64) | int(b) for a, b in zip(hi, lo)]
    assert all(a < b for a, b in zip(k, k[1:])) and counts.sum() == raw.shape[0]


def test_dedup_empty():
    keys, counts = oracle.dedup(np.zeros((0, 2), dtype=np.uint64))
    assert keys.shape == (0, 2) and counts.shape == (0,)
