"""Host-side pieces of bench.py: the kernel counts it claims, and the source hash that ties a
committed ncu capture to the code it was taken on."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_plain_launch_counts():
    b = _bench()
    # table build, main kernel, two reduction passes
    assert b._plain_launches({"kernel": 2}, 1000) == 4
    assert b._plain_launches({"kernel": 3}, 10 ** 6) == 4
    # with the join at 1e5 rows: sets of 2^18 slots, keys up to 2^20 -> two 11-bit passes:
    # group-start scan 3 + 2 x (hist + scan 3 + scatter) + gather + mark + order (key + 5)
    assert b._plain_launches({"kernel": 4}, 100_000) == 4 + 3 + 10 + 2 + 6
    # against a caller's table the samples' group sizes are looked up first
    assert b._plain_launches({"kernel": 4}, 100_000, caller_table=True) == 4 + 3 + 10 + 2 + 6 + 1
    # 2^20 slots per set (5e5 rows): keys up to 2^21 (22 bits) -> still two passes;
    # 2^21 slots (1e6 rows): keys up to 2^22 (23 bits) -> three
    assert b._plain_launches({"kernel": 5}, 500_000) == 25
    assert b._plain_launches({"kernel": 5}, 1_000_000) == 30


def test_batched_launch_counts():
    b = _bench()
    small = [{"n_u": 1000}, {"n_u": 5000}]
    assert b._batched_launches(small) == 4          # no molecule takes the join
    big = small + [{"n_u": 20000}, {"n_u": 100000}]
    n = b._batched_launches(big)
    # one shared index (two or three passes, gather, mark), then the order of four molecules'
    # rows: a key kernel and one pass over keys up to (4 << 8) | 255 (11 bits)
    assert n in (4 + 3 + 10 + 2 + 6, 4 + 3 + 15 + 2 + 6)
    # 64 molecules: keys up to (64 << 8) | 255 (15 bits) -> two order passes
    many = big + [{"n_u": 1000}] * 60
    assert b._batched_launches(many) - b._batched_launches(big) == 5


def test_source_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    b = _bench()
    csrc = tmp_path / "paper_2506_23809_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("qc_kernels.cu", "qc_main_kernel.cuh", "qc_device.cuh", "qc_internal.h"):
        shutil.copy(os.path.join(ROOT, "paper_2506_23809_gb300", "csrc", f), csrc / f)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    h0 = b._source_hash()
    dev = csrc / "qc_device.cuh"
    text = dev.read_text()
    dev.write_text("// a new comment line\n/* and a block\n   comment */\n" + text.replace("\n", "\n  ", 3))
    assert b._source_hash() == h0
    dev.write_text(text.replace("kCandCap = 160", "kCandCap = 192", 1))
    assert b._source_hash() != h0


def test_work_l2_bytes_formula():
    """The roofline's algorithmic bytes from counted work, term by term (N=52, 14 e: o = 7,
    v = 19, 2 o v = 266 spin-string lookups per sample; FP64 elements)."""
    b = _bench()
    zero = dict(samples=0, scan_rows=0, tests=0, probes=0, hits_single=0, hits_same=0, hits_ab=0, ctas=0,
                hits_scanned=0, beta_looked=0, beta_groups=0)
    assert b.work_l2_bytes(zero, 14, 52, 8, 14) == 0
    cases = [("scan_rows", 16), ("probes", 16), ("hits_single", 32 + 8 * 22), ("hits_same", 48), ("hits_ab", 40),
             ("samples", 48 + 8 * 266), ("ctas", 4 << 14), ("tests", 0), ("hits_scanned", -16),
             ("beta_looked", 8), ("beta_groups", 0)]
    for k, per in cases:
        w = dict(zero)
        w[k] = 3
        assert b.work_l2_bytes(w, 14, 52, 8, 14) == 3 * per, k
    w = dict(zero, hits_single=1, hits_same=1, hits_ab=1)
    assert b.work_l2_bytes(w, 20, 76, 4, 15) == (32 + 4 * 31) + (32 + 8) + (32 + 4)
