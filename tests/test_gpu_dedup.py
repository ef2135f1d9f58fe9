"""The sample table built on the device (qc_dedup) against the oracle: bit-exact keys and
multiplicities for random streams (ragged sizes, 14 to 128 significant bits, many repeats),
the round trip of an expanded sample set into qc_eloc_eval, and the error cases."""
import random

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


def _stream(n, n_bits, seed, distinct):
    rnd = random.Random(seed)
    pool = [rnd.getrandbits(n_bits) for _ in range(distinct)]
    vals = [rnd.choice(pool) for _ in range(n)]
    return np.array([[v & ((1 << 64) - 1), v >> 64] for v in vals], dtype=np.uint64).reshape(-1, 2)


def _gpu(B, raw, n_orb):
    import torch
    t = torch.from_numpy(raw.view(np.int64).copy()).cuda()
    k, c, u = B.qc_dedup(t, n_orb)
    torch.cuda.synchronize()
    n = int(u.item())
    if n < 0:
        return None, None, n
    return k[:n].cpu().numpy().view(np.uint64), c[:n].cpu().numpy(), n


@pytest.mark.parametrize("n,n_bits,distinct", [(1, 14, 1), (1000, 14, 300), (5000, 52, 900), (100003, 52, 20000),
                                               (70001, 70, 5000), (40000, 128, 39000), (9000, 8, 256)])
def test_dedup_equals_oracle(B, orc, n, n_bits, distinct):
    import oracle
    raw = _stream(n, n_bits, 17 + n + n_bits, distinct)
    keys, counts, u = _gpu(B, raw, n_bits)
    wk, wc = oracle.dedup(raw)
    assert u == wk.shape[0]
    assert np.array_equal(keys, wk) and np.array_equal(counts, wc)


def test_dedup_round_trip_into_eval(B, orc):
    """A seeded sample set expanded by its counts and shuffled dedups back to exactly that
    set, and evaluating the device-built table gives bitwise the same E_loc."""
    import torch
    ints, s = I.make_workload("n14_e6_u1k")
    rng = np.random.default_rng(3)
    raw = np.repeat(s.keys, s.counts, axis=0)
    raw = raw[rng.permutation(raw.shape[0])]
    keys, counts, u = _gpu(B, raw, 14)
    assert np.array_equal(keys, s.keys) and np.array_equal(counts, s.counts)
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, 14, 6)
    try:
        p = torch.from_numpy(s.psi).cuda()
        e1, _ = B.qc_eloc_eval(h, B.keys_to_tensor(s.keys), torch.from_numpy(s.counts).cuda(), p)
        e1 = e1.cpu().numpy()
        e2, _ = B.qc_eloc_eval(h, B.keys_to_tensor(keys), torch.from_numpy(counts).cuda(), p)
        assert np.array_equal(e1.view(np.uint64), e2.cpu().numpy().view(np.uint64))
    finally:
        B.qc_eloc_destroy(h)


def test_dedup_errors(B):
    import torch
    raw = _stream(100, 20, 5, 30)
    raw[7, 0] |= np.uint64(1 << 40)            # a bit beyond n_orb = 20
    assert _gpu(B, raw, 20)[2] == -1
    empty = torch.zeros((0, 2), dtype=torch.int64, device="cuda")
    _, _, u = B.qc_dedup(empty, 20)
    assert int(u.item()) == 0
    t = torch.from_numpy(_stream(1000, 20, 6, 100).view(np.int64).copy()).cuda()
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    import ctypes
    with pytest.raises(B.QcError):   # a workspace that is too small is refused before any work
        st = B.load_library().qc_dedup(ctypes.c_void_p(t.data_ptr()), 1000, 20,
                                       ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                       ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(small.data_ptr()), 1024,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        B._check(st, None)
