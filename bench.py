#!/usr/bin/env python
"""Benchmark of the sample-space local-energy step (Eq. 5) and its reduction (Eq. 1).

One step = one qc_eloc_eval over the whole workload: hash-index + Bloom-filter build over
the unique-sample table, the local-energy kernel (every single and double excitation of
every sample, looked up in the table), and the two-pass count-weighted reduction.

Workload (default): N = 52 spin orbitals, 14 electrons, 1e5 unique rank-weighted samples
with Zipf(1.2) counts summing to 1e7, complex FP64 psi, FP64 arithmetic; synthetic seeded
integrals (h: -U(1,5) diagonal, N(0, 0.1 e^{-|p-q|/2}) off-diagonal; (pq|rs) from a rank-52
Cholesky-like factor).  25,137 connected pairs per sample, 2.51e9 per step.

With N GPUs (torchrun) the unique-sample set grows to N x 1e5 (weak scaling); rank r
evaluates rows [r*1e5, (r+1)*1e5) against the whole table, and the per-rank partial sums
of Eq. 1 are combined on the host (the MPI_Allreduce of Alg. 3).

``--impl reference`` times the CPU oracle instead (rank 0 only), on bounded samples of the
same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "connected matrix elements/sec and E_loc samples/sec vs L2/HBM roofline; serve p50/p99"
UNIT = "connected matrix elements/s"
# The roofline of the local-energy kernel is computed from the work it did in one launch,
# counted on the device (QC_OPT_COUNT_WORK, one untimed evaluation after the timed steps):
#   ALU operations = 7 x filter tests: form the excitation's hash (1 XOR), derive the filter
#     word offset (1), shift the word to its three bit positions (3), combine (1), test (1);
#     the word itself is read through the load/store pipe and is not counted;
#   L2 bytes = 16 per scanned table row (the join's entry) + 16 per bucket probe
#     + per hit 16 (psi(x')) + 16 (the stored key, which a hit found by the join's scan does not
#     load: its entry already matched) + its integrals, e bytes each (8 FP64, 4 FP32):
#       single 1 + 3 n_elec / 2 (h_ai, (ai|kk) over the occupied k, (ak|ki) over the same spin),
#       same-spin double 2, opposite-spin double 1
#     + per sample 16 (x) + 16 (psi(x)) + 16 (E_loc written) + 8 per spin-string set lookup
#       (one per single excitation, 2 o v, and one per beta' the join's beta' phase classifies)
#     + per CTA the Bloom filter copied into shared memory (4 x 2^fw).
# achieved = that work / the kernel's mean event-timed duration over the timed steps; the
# peaks are the derived ALU peak (SMs x 4 x 16 lanes x max clock) with the library's measured
# ALU probe beside it, and the measured L2 gather probe (random 16-byte loads from an
# L2-resident table).  The resource with the larger fraction is reported as the bound.
OPS_PER_TEST = 7
# Lanes of the integer ALU pipe per SM sub-partition.  ncu reports the ALU pipe at 61.4 %
# of its peak while the SM issues 2.44 of 4 instructions per cycle: a 32-lane pipe would
# need more ALU instructions than were issued in total, so the pipe is 16 lanes wide
# (a warp instruction every other cycle).
ALU_LANES = 16
# Nominal dense FP64 rate of the part, GFLOP/s (the gradient contraction's bound).
FP64_NOMINAL_GFLOPS = 1250.0
PROFILE_DIR = os.path.join(ROOT, "profiles")  # eloc_main_<workload>.json: ncu counters of the main kernel


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="n52_e14_u100k")
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32c"])
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--form", default="plain", choices=["plain", "batched", "serve", "grad", "dedup", "full", "sweep"],
                   help="plain: one molecule per step (the default benchmark); batched: many "
                        "molecules in one persistent launch; serve: Poisson request arrivals")
    p.add_argument("--n-mol", type=int, default=64, help="batched form: molecules")
    p.add_argument("--systems", default="", help="sweep form: comma-separated subset of the paper's systems")
    p.add_argument("--n-par", type=int, default=4096, help="grad form: parameters (columns of d ln Psi*)")
    p.add_argument("--chunk", type=int, default=10000, help="full form: samples per export/apply chunk")
    p.add_argument("--requests", type=int, default=48, help="serve form: requests")
    p.add_argument("--serve-traces", type=int, default=3,
                   help="serve form: seeded arrival traces per rate (the first is the specs' own)")
    p.add_argument("--wave-rows", type=int, default=-1,
                   help="serve form: QC_SRV_OPT_WAVE_ROWS (-1: the library's default)")
    p.add_argument("--rates", default="", help="serve form: comma-separated arrival rates per second "
                                                "(default: 0.3, 0.7 and 1.5 x the plain capacity)")
    p.add_argument("--quantum", type=float, default=1e12,
                   help="serve form: enumerated pairs per wave (0: one wave takes every ready request)")
    p.add_argument("--oldest-pct", type=int, default=50,
                   help="serve form: percent of a wave guaranteed to the oldest request")
    return p.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _plain_launches(cfg, n_table, caller_table=False):
    """Kernels of one plain evaluation: table build, main kernel, two reduction passes, and
    with the sample-space join its index: a 3-kernel scan of the group sizes, per 11-bit
    radix pass a histogram, a 3-kernel scan and a scatter, the gather and the mark pass, and
    the heavy-first sample order (a key kernel and one radix pass; against a caller's table,
    first a look-up of the samples' group sizes)."""
    n = 4
    if cfg["kernel"] in (4, 5):
        size = 1 << max(0, (2 * max(n_table, 1) - 1).bit_length())  # hash sets: next_pow2(2n) slots
        passes = -(-(2 * size).bit_length() // 11)
        n += 3 + 5 * passes + 2 + 6 + (1 if caller_table else 0)
    return n


def _batched_launches(specs):
    """Kernels of one batched step: the batch build, the batch kernel and two reduction
    passes, and for the molecules that take the join (join_by_default: 16384 rows up, or 2e8
    rows x pairs per sample, or 512 rows at 50000 pairs per sample) one shared index: a
    3-kernel scan, per 11-bit radix pass a histogram, a 3-kernel scan and a scatter, the
    gather and the mark pass; then the rows heavy first, molecule by molecule: a key kernel
    and one radix sort of keys up to (molecules << 8) | 255."""
    n = 4

    def joins(sp):
        p = _pairs(sp["n_orb"], sp["n_elec"]) if "n_orb" in sp else 0
        return sp["n_u"] >= 16384 or sp["n_u"] * p >= 200_000_000 or (p >= 50_000 and sp["n_u"] >= 512)
    slots = sum(2 * (1 << max(0, (2 * sp["n_u"] - 1).bit_length())) for sp in specs if joins(sp))
    if slots:
        n += 3 + 5 * (-(-slots.bit_length() // 11)) + 2
        n += 1 + 5 * (-(-((len(specs) << 8) | 255).bit_length() // 11))
    return n


def _source_hash():
    """Hash of the main kernel's sources without their comments and whitespace: a profile's
    counters stay attached to the code they were taken on, not to its comments."""
    import re
    h = hashlib.sha256()
    for f in ("qc_kernels.cu", "qc_main_kernel.cuh", "qc_device.cuh", "qc_internal.h"):
        with open(os.path.join(ROOT, "paper_2506_23809_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the GPU runs."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                sm.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for n, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        busy = [v for v in sm if mx is None or v >= 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _make_workload(name, world):
    from paper_2506_23809_gb300 import inputs as I
    spec = dict(I.WORKLOADS[name])
    kind, total = spec["counts"]
    return spec, I.make_workload(n_orb=spec["n_orb"], n_elec=spec["n_elec"], rank=spec["rank"],
                                 n_u=spec["n_u"] * world, sampler=spec["sampler"],
                                 counts=(kind, total * world), seed=spec["seed"])


def work_l2_bytes(w, n_elec, n_orb, elem_bytes, filter_log2w):
    """Algorithmic L2 bytes of one local-energy launch from its work counts (see the table at
    the top of this file)."""
    o = n_elec // 2
    v = n_orb // 2 - o
    return (16 * w["scan_rows"] + 16 * w["probes"]
            + (32 + elem_bytes * (1 + 3 * n_elec // 2)) * w["hits_single"]
            + (32 + 2 * elem_bytes) * w["hits_same"] + (32 + elem_bytes) * w["hits_ab"]
            + (48 + 8 * 2 * o * v) * w["samples"] + (4 << filter_log2w) * w["ctas"]
            - 16 * w.get("hits_scanned", 0) + 8 * w.get("beta_looked", 0))


def _cpu_baseline(ints, s, spec, target_s, pairs_per_sample, gpu_eloc=None):
    """The oracle, as it stands, on a bounded seeded sample of rows (each looks its
    excitations up in the whole table), all host cores.  With gpu_eloc, also the error of
    the GPU's E_loc against the oracle's on those rows."""
    import numpy as np
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(12345)
    perm = rng.permutation(s.n_u)

    last = {}

    def run(rows, threads):
        sel = np.sort(perm[:rows])
        t = time.perf_counter()
        e = oracle.eloc(ints.h, ints.eri, 0.0, spec["n_orb"], s.keys[sel], s.psi[sel], s.keys, s.psi,
                        nthreads=threads)
        dt = time.perf_counter() - t
        last["sel"], last["eloc"] = sel, e
        return dt

    probe = min(s.n_u, 4 * cores)
    t0 = run(probe, cores)
    rows = int(min(s.n_u, max(probe, probe * target_s / max(t0, 1e-6))))
    t1 = run(rows, cores)
    err = None
    if gpu_eloc is not None:
        d = np.abs(gpu_eloc[last["sel"]] - last["eloc"])
        err = {"rows": int(rows), "max_abs_ha": float(d.max()), "rms_abs_ha": float(np.sqrt((d ** 2).mean())),
               "max_rel": float((d / np.maximum(1.0, np.abs(last["eloc"]))).max())}
    # one thread, on a sample sized for about a tenth of the all-core time
    rows1 = int(min(s.n_u, max(4, rows * 0.1 / cores)))
    t2 = run(rows1, 1)
    out = {"value": rows * pairs_per_sample / t1, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{rows} seeded random rows of the {s.n_u}-row table (all rows looked up in the "
                     f"whole table), {t1:.1f} s on {cores} threads; single thread: {rows1} rows, {t2:.2f} s",
           "samples_per_s": rows / t1, "value_1_thread": rows1 * pairs_per_sample / t2}
    return out, err


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.build()
    spec, (ints, s) = _make_workload(args.workload, 1)
    K, N = spec["n_orb"] // 2, spec["n_elec"] // 2
    o, v = N, K - N
    pairs = 2 * o * v + 2 * (o * (o - 1) // 2) * (v * (v - 1) // 2) + (o * v) ** 2
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(777)
    # size one step to ~2 s of oracle work
    probe = 4 * cores
    sel = np.sort(rng.choice(s.n_u, probe, replace=False))
    t = time.perf_counter()
    oracle.eloc(ints.h, ints.eri, 0.0, spec["n_orb"], s.keys[sel], s.psi[sel], s.keys, s.psi, nthreads=cores)
    dt = time.perf_counter() - t
    rows = int(min(s.n_u, max(probe, probe * 2.0 / max(dt, 1e-6))))
    steps = []
    for i in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(s.n_u, rows, replace=False))
        t = time.perf_counter()
        el = oracle.eloc(ints.h, ints.eri, 0.0, spec["n_orb"], s.keys[sel], s.psi[sel], s.keys, s.psi,
                         nthreads=cores)
        oracle.reduce(el, s.counts[sel])
        if i >= args.warmup:
            steps.append(time.perf_counter() - t)
    total = sum(steps)
    value = rows * pairs * len(steps) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": args.workload, "n_orb": spec["n_orb"], "n_elec": spec["n_elec"],
                       "n_u": spec["n_u"], "pairs_per_sample": pairs, "rows_per_step": rows,
                       "mode": "sample"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{rows} seeded random rows per step of the {s.n_u}-row table"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build, shards

    world, rank, local = _dist()
    build.build()
    B.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    spec, (ints, s) = _make_workload(args.workload, world)
    lo, hi = shards.shard_rows(s.n_u, world, rank)
    n_rank = hi - lo
    prec = B.QC_FP64 if args.precision == "fp64" else B.QC_FP32_COMP
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, spec["n_orb"], spec["n_elec"], prec, B.QC_SAMPLE)
    B.qc_eloc_set_option(h, B.QC_OPT_TIMING, 1)
    pairs_per_sample = B.qc_eloc_pairs_per_sample(h)

    keys_all = B.keys_to_tensor(s.keys, dev)
    psi_all = torch.from_numpy(s.psi).to(dev)
    cnt_all = torch.from_numpy(s.counts).to(dev)
    keys, psi, cnt = keys_all[lo:hi], psi_all[lo:hi], cnt_all[lo:hi]
    tk, tp = (keys_all, psi_all) if world > 1 else (None, None)
    eloc = torch.empty(n_rank, dtype=torch.complex128, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)
    B.qc_eloc_reserve(h, n_rank, s.n_u)

    enqueue_s = []

    def step():
        t = time.perf_counter()
        B.qc_eloc_eval(h, keys, cnt, psi, tk, tp, eloc=eloc, stream=stream)
        enqueue_s.append(time.perf_counter() - t)

    # the clock sampler starts before the warm-up, which keeps the GPU busy (no idle gap, so
    # no clock ramp-up inside the timed region) and gives the sampler its first samples
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    enqueue_s.clear()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    step_ms, main_ms, table_ms, red_ms, host_ms = [], [], [], [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    for k in range(args.steps):
        t_h = time.perf_counter()
        flush.fill_(float(k))
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        t3 = B.qc_eloc_timings(h)
        host_ms.append(1e3 * (time.perf_counter() - t_h))
        table_ms.append(t3[0])
        main_ms.append(t3[1])
        red_ms.append(t3[2])
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    wall = time.perf_counter() - t_wall
    sampler.stop()
    summ = B.qc_eloc_summary_read(h, stream)
    cfg = B.qc_eloc_last_config(h)

    total_s = sum(step_ms) / 1e3
    pairs_rank = int(summ["n_pairs"])
    t_max, pairs_all, samples_all = total_s, pairs_rank, n_rank
    if pg:
        v = torch.tensor([total_s], dtype=torch.float64, device=dev)
        pg.all_reduce(v, op=pg.ReduceOp.MAX)
        t_max = float(v.item())
        c = torch.tensor([pairs_rank, n_rank], dtype=torch.float64, device=dev)
        pg.all_reduce(c)
        pairs_all, samples_all = int(c[0].item()), int(c[1].item())
        # Eq. 1 across ranks: gather (W, sum cE, W * var) and combine
        W, Ebar, var = shards.allgather_combine(shards.partials(summ), pg, device=dev, status=int(summ["status"]))
    else:
        W, Ebar, var = summ["w"], summ["energy"], summ["var"]
    value = pairs_all * args.steps / t_max
    samples_per_s = samples_all * args.steps / t_max

    # ---- end to end through the C ABI from page-locked host buffers ----
    e2e = None
    if not args.no_e2e:
        keys_h = torch.from_numpy(s.keys[lo:hi].view(np.int64)).pin_memory()
        psi_h = torch.from_numpy(s.psi[lo:hi]).pin_memory()
        cnt_h = torch.from_numpy(s.counts[lo:hi]).pin_memory()
        eloc_h = torch.empty(n_rank, dtype=torch.complex128).pin_memory()
        keys_d, psi_d, cnt_d = torch.empty_like(keys), torch.empty_like(psi), torch.empty_like(cnt)
        h2d = keys_h.numel() * 8 + psi_h.numel() * 16 + cnt_h.numel() * 8
        if world > 1:
            tk_h = torch.from_numpy(s.keys.view(np.int64)).pin_memory()
            tp_h = torch.from_numpy(s.psi).pin_memory()
            tk_d, tp_d = torch.empty_like(keys_all), torch.empty_like(psi_all)
            h2d += tk_h.numel() * 8 + tp_h.numel() * 16
        d2h = eloc_h.numel() * 16 + 96

        def e2e_step():
            keys_d.copy_(keys_h, non_blocking=True)
            psi_d.copy_(psi_h, non_blocking=True)
            cnt_d.copy_(cnt_h, non_blocking=True)
            a, b = None, None
            if world > 1:
                tk_d.copy_(tk_h, non_blocking=True)
                tp_d.copy_(tp_h, non_blocking=True)
                a, b = tk_d, tp_d
            B.qc_eloc_eval(h, keys_d, cnt_d, psi_d, a, b, eloc=eloc, stream=stream)
            eloc_h.copy_(eloc, non_blocking=True)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        e_ms, e_host = [], []
        for k in range(args.steps):
            flush.fill_(float(k))
            stream.synchronize()
            t_h = time.perf_counter()
            ev0.record(stream)
            e2e_step()
            ev1.record(stream)
            ev1.synchronize()        # the caller can use E_loc from here on
            e_host.append(time.perf_counter() - t_h)
            e_ms.append(ev0.elapsed_time(ev1))
        et = sum(e_ms) / 1e3
        if pg:
            v = torch.tensor([et], dtype=torch.float64, device=dev)
            pg.all_reduce(v, op=pg.ReduceOp.MAX)
            et = float(v.item())
        e2e = {"value": pairs_all * args.steps / et, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * et / args.steps,
               # host wall clock from the first copy's enqueue to E_loc usable on the host
               "host_ms_per_step": 1e3 * statistics.median(e_host)}

    # ---- roofline of the dominant kernel (the local-energy kernel), from counted work ----
    peaks, peak_src = _measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 4 * ALU_LANES * sm_max * 1e6  # ALU pipe, ops/s (derived)
    main_s = statistics.mean(main_ms) / 1e3
    B.qc_eloc_set_option(h, B.QC_OPT_COUNT_WORK, 1)
    B.qc_eloc_eval(h, keys, cnt, psi, tk, tp, eloc=eloc, stream=stream)   # untimed: counts the work
    work = B.qc_eloc_work(h)
    B.qc_eloc_set_option(h, B.QC_OPT_COUNT_WORK, 0)
    elem = 8 if prec == B.QC_FP64 else 4
    ops = OPS_PER_TEST * work["tests"]
    l2_bytes = work_l2_bytes(work, spec["n_elec"], spec["n_orb"], elem, cfg["filter_log2w"])
    traffic = issue = None
    profile_json = os.path.join(PROFILE_DIR, f"eloc_main_{args.workload}.json")
    if os.path.exists(profile_json):
        with open(profile_json) as f:
            prof = json.load(f)
        if prof.get("source_hash") == _source_hash() and prof.get("workload") == args.workload:
            traffic = prof.get("dram_bytes_per_launch")
            issue = prof.get("issue_active_frac")
    probe = {}
    try:  # measured ceilings (probes of the library, after the timed region)
        probe = B.qc_probe_peaks()
    except Exception as ex:  # noqa: BLE001 -- a probe failure must not lose the bench line
        probe = {"error": str(ex)}
    l2_peak = probe.get("l2_gather_gbs")
    alu = {"ops": ops, "achieved_gops": ops / main_s / 1e9, "peak_gops": peak_ops / 1e9,
           "frac": ops / main_s / peak_ops,
           "peak_basis": f"{props.multi_processor_count} SMs x 4 sub-partitions x {ALU_LANES} ALU lanes x "
                         f"{sm_max:.0f} MHz ({peak_src} sm_max_mhz)",
           "probe_gops": probe.get("alu_ops_per_s", 0.0) / 1e9 or None}
    l2 = {"bytes": l2_bytes, "achieved_gbs": l2_bytes / main_s / 1e9, "peak_gbs": l2_peak,
          "frac": (l2_bytes / main_s / 1e9 / l2_peak) if l2_peak else None,
          "peak_basis": "measured: qc_probe_peaks random 16-byte loads from a 4 MB L2-resident table"}
    use_l2 = l2["frac"] is not None and l2["frac"] > alu["frac"]
    roofline = {"bound": "l2" if use_l2 else "alu",
                "achieved": l2["achieved_gbs"] if use_l2 else alu["achieved_gops"],
                "peak": l2["peak_gbs"] if use_l2 else alu["peak_gops"],
                "unit": "GB/s" if use_l2 else "Gop/s",
                "frac": l2["frac"] if use_l2 else alu["frac"], "traffic": traffic,
                "kernel": {1: "eloc_main_kernel (unfiltered)", 2: "eloc_main_kernel (filtered)",
                           3: "eloc_main_kernel (filtered, lean lists)",
                           4: "eloc_main_kernel (sample-space join)",
                           5: "eloc_main_kernel (sample-space join, lean lists)"}.get(cfg["kernel"], "eloc_main_kernel"),
                "kernel_ms": 1e3 * main_s, "counted_work": work, "alu": alu, "l2": l2,
                "formula": "alu: 7 x tests; l2: bench.work_l2_bytes(counted_work); achieved = work / kernel_ms",
                "hbm_peak_gbs": peaks.get("hbm_gbs"),
                # ncu's share of issue slots that issued (same kernel sources): the kernel is
                # bound by issue and latency rather than by either unit
                "issue_active_frac": issue}

    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, err = _cpu_baseline(ints, s, spec, args.cpu_seconds, pairs_per_sample, eloc.cpu().numpy())

    clocks = sampler.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == B.QC_FP64 else "f32+f64",
            "data": "synthetic (seeded integrals, rank-weighted unique samples, Zipf counts, lognormal psi)",
            "config": {"workload": args.workload, "n_orb": spec["n_orb"], "n_elec": spec["n_elec"],
                       "n_u_per_gpu": n_rank, "n_table": int(s.n_u), "pairs_per_sample": pairs_per_sample,
                       "counts_total": int(s.counts.sum()), "mode": "sample", "precision": args.precision,
                       "l2": "256 MB buffer written between timed steps", "parallelism": f"samples x{world}",
                       "launch": cfg},
            "samples_per_s": samples_per_s,
            "energy": {"re": Ebar.real, "im": Ebar.imag, "var": var, "w": W},
            "phase_ms": {"table": statistics.mean(table_ms), "main": statistics.mean(main_ms),
                         "reduce": statistics.mean(red_ms)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": _plain_launches(cfg, int(s.n_u), caller_table=world > 1) * args.steps, "clocks": clocks,
            "wall_s_timed": wall,
            # host wall clock of one timed step (flush, enqueue, wait, phase timings) and of the
            # qc_eloc_eval call alone (argument checks, launch set-up, enqueue)
            "host_ms_per_step": 1e3 * wall / args.steps, "host_ms_step_median": statistics.median(host_ms),
            "host_ms_step_max": max(host_ms), "enqueue_ms": 1e3 * statistics.median(enqueue_s),
            "error_vs_oracle": err,
            "value_basis": "structural connected pairs: samples x pairs per sample (every S_z-conserving "
                           "single and double), however the kernel resolves them",
            "hits_per_step": int(summ["n_hits"]), "status": int(summ["status"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.qc_eloc_destroy(h)
    if pg:
        pg.destroy_process_group()
    return 0


def _pairs(n_orb, n_elec):
    K, o = n_orb // 2, n_elec // 2
    v = K - o
    return 2 * o * v + 2 * (o * (o - 1) // 2) * (v * (v - 1) // 2) + (o * v) ** 2


def run_batched(args):
    """64 synthetic molecules (N even in 24..120, FP32-compensated): plain per-molecule
    launches against one batched step, eager and as an autotuned CUDA graph."""
    import numpy as np
    import torch

    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    from paper_2506_23809_gb300 import inputs as I
    build.build()
    B.load_library()
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    specs = I.batched_molecule_specs(args.n_mol)
    # the batched form computes in the precision form (FP32 terms, compensated sums, FP64
    # diagonal and reduction) unless --precision fp64 is given explicitly
    prec = B.QC_FP64 if "--precision" in sys.argv and args.precision == "fp64" else B.QC_FP32_COMP
    if world > 1:
        return _run_batched_plan(args, specs, prec, world, rank, local)
    handles, dev, outs = [], [], []
    total_pairs = 0
    for sp in specs:
        K = sp["n_orb"] // 2
        ints = I.make_integrals(K, sp["n_orb"], sp["seed"])
        keys = I.rank_weighted_samples(K, sp["n_elec"] // 2, sp["n_elec"] // 2, sp["n_u"], seed=sp["seed"] + 1)
        counts = I.zipf_counts(sp["n_u"], 100 * sp["n_u"], sp["seed"] + 2)
        psi = I.lognormal_psi(sp["n_u"], sp["seed"] + 3)
        h = B.qc_eloc_create(ints.h, ints.eri, 0.0, sp["n_orb"], sp["n_elec"], prec)
        B.qc_eloc_set_option(h, B.QC_OPT_TIMING, 1)
        handles.append(h)
        dev.append((B.keys_to_tensor(keys), torch.from_numpy(counts).cuda(), torch.from_numpy(psi).cuda()))
        outs.append(torch.empty(sp["n_u"], dtype=torch.complex128, device="cuda"))
        total_pairs += sp["n_u"] * _pairs(sp["n_orb"], sp["n_elec"])
    stream = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        stream.synchronize()
        ts = []
        for _ in range(reps):
            ev0.record(stream)
            fn()
            ev1.record(stream)
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1))
        return statistics.median(ts)

    def plain():
        for h, (k, c, p), o in zip(handles, dev, outs):
            B.qc_eloc_eval(h, k, c, p, eloc=o, stream=stream)
    with torch.cuda.stream(stream):
        t_plain = timed(plain, args.steps)
        ref = [o.cpu().numpy().copy() for o in outs]
        batch = B.qc_batch_create(handles)
        for m, ((k, c, p), o) in enumerate(zip(dev, outs)):
            B.qc_batch_set_inputs(batch, m, k, c, p, o)
        t_eager = timed(lambda: B.qc_batch_eval(batch, stream), args.steps)
        best = B.qc_batch_autotune(batch, stream, iters=2)
        t_tuned = timed(lambda: B.qc_batch_eval(batch, stream), args.steps)
        t_graph = timed(lambda: B.qc_batch_graph_launch(batch, stream), args.steps)
        # the two paths may pick different filter sizes, which changes the order hits are
        # summed in: compare within the precision form's tolerance
        diff = max(float(np.max(np.abs(o.cpu().numpy() - r) / np.maximum(1.0, np.abs(r)), initial=0.0))
                   for o, r in zip(outs, ref))
        cfg = B.qc_batch_config(batch)
    B.qc_batch_destroy(batch)
    for h in handles:
        B.qc_eloc_destroy(h)
    line = {"metric": METRIC, "form": "batched", "value": total_pairs / (t_graph / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_graph,
            "higher_is_better": True, "dtype": "f32+f64" if prec == B.QC_FP32_COMP else "f64",
            "config": {"workload": f"batched_{args.n_mol}_molecules", "n_mol": args.n_mol,
                       "total_samples": int(sum(sp["n_u"] for sp in specs)), "pairs_per_step": int(total_pairs),
                       "n_orb_range": [min(sp["n_orb"] for sp in specs), max(sp["n_orb"] for sp in specs)],
                       "autotuned": best, "launch": cfg},
            "ms": {"plain_per_molecule_launches": t_plain, "batched_eager": t_eager,
                   "batched_eager_autotuned": t_tuned, "batched_graph_autotuned": t_graph},
            "speedup_vs_plain": t_plain / t_graph, "max_rel_diff_vs_plain": diff,
            "gpu_launches": _batched_launches(specs) * args.steps}
    print(json.dumps(line), flush=True)
    return 0


def _batched_molecule(I, sp):
    K = sp["n_orb"] // 2
    ints = I.make_integrals(K, sp["n_orb"], sp["seed"])
    keys = I.rank_weighted_samples(K, sp["n_elec"] // 2, sp["n_elec"] // 2, sp["n_u"], seed=sp["seed"] + 1)
    return ints, keys, I.zipf_counts(sp["n_u"], 100 * sp["n_u"], sp["seed"] + 2), I.lognormal_psi(sp["n_u"], sp["seed"] + 3)


def _run_batched_plan(args, specs, prec, world, rank, local):
    """The batched workload over N GPUs with a cost-weighted plan (Alg. 2's split with
    measured costs): rank 0 times every molecule once and spreads that over its rows by hit
    count, the plan (row ranges of molecules per rank) is broadcast, and each rank runs its
    pieces as one batched step (autotuned, replayed as a CUDA graph).  The pieces' Eq. 1
    partials are gathered and combined per molecule: 32 bytes per piece, the one exchange."""
    import torch
    import torch.distributed as dist

    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import inputs as I
    from paper_2506_23809_gb300 import shards
    dev = torch.device("cuda", local)
    dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream()
    plan = [None]
    if rank == 0:
        handles, inputs = [], []
        for sp in specs:
            ints, keys, counts, psi = _batched_molecule(I, sp)
            handles.append(B.qc_eloc_create(ints.h, ints.eri, 0.0, sp["n_orb"], sp["n_elec"], prec))
            inputs.append((B.keys_to_tensor(keys, dev), torch.from_numpy(counts).to(dev), torch.from_numpy(psi).to(dev),
                           torch.empty(sp["n_u"], dtype=torch.complex128, device=dev)))
        with torch.cuda.stream(stream):
            costs = shards.calibrate_row_costs(B, handles, inputs, stream)
        plan = [shards.plan_pieces(costs, world)]
        for h in handles:
            B.qc_eloc_destroy(h)
        del inputs
    dist.broadcast_object_list(plan, src=0)
    plan = plan[0]
    mine = plan[rank]
    mols = sorted({m for m, _, _ in mine})
    handles, inputs = {}, {}
    for m in mols:
        sp = specs[m]
        ints, keys, counts, psi = _batched_molecule(I, sp)
        handles[m] = B.qc_eloc_create(ints.h, ints.eri, 0.0, sp["n_orb"], sp["n_elec"], prec)
        inputs[m] = (B.keys_to_tensor(keys, dev), torch.from_numpy(counts).to(dev), torch.from_numpy(psi).to(dev),
                     torch.empty(sp["n_u"], dtype=torch.complex128, device=dev))
    with torch.cuda.stream(stream):
        batch, _ = shards.evaluate_pieces(B, handles, inputs, mine, stream, autotune=True, graph=True)
        for _ in range(args.warmup):
            B.qc_batch_graph_launch(batch, stream)
        stream.synchronize()
        dist.barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            B.qc_batch_graph_launch(batch, stream)
        ev1.record(stream)
        ev1.synchronize()
        sums = B.qc_batch_summaries(batch, stream)
    t = torch.tensor([ev0.elapsed_time(ev1) / args.steps], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    parts = [(m, shards.partials(sm)) for (m, _, _), sm in zip(mine, sums)]
    gathered = [None] * world
    dist.all_gather_object(gathered, parts)
    energies = shards.combine_pieces(len(specs), [x for g in gathered for x in g])
    B.qc_batch_destroy(batch)
    for h in handles.values():
        B.qc_eloc_destroy(h)
    total_pairs = sum(sp["n_u"] * _pairs(sp["n_orb"], sp["n_elec"]) for sp in specs)
    ms = float(t.item())
    if rank == 0:
        line = {"metric": METRIC, "form": "batched", "value": total_pairs / (ms / 1e3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "dtype": "f32+f64" if prec == B.QC_FP32_COMP else "f64",
                "config": {"workload": f"batched_{len(specs)}_molecules", "parallelism": f"cost-weighted plan x{world}",
                           "pieces_per_rank": [len(p) for p in plan]},
                "energy_checksum": float(sum(E.real for _, E, _ in energies)),
                "gpu_launches": None}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def run_serve(args):
    """Poisson arrivals of requests with their own molecules (the serving spec: N even in
    28..128, half filling +-4 electrons, lognormal unique-sample counts clipped to 1e3..1e6,
    rank-N integrals), at three arrival rates set against the measured capacity of plain
    per-request evaluation (the last above it, so the GPU saturates).  Two arms see the same
    arrivals: the server (continuous batching) and a live plain FIFO -- one worker thread that
    creates a handle, uploads, evaluates, reads E_loc back and destroys the handle, request
    after request in arrival order.  Latency = completion - arrival; sustained throughput =
    the requests' structural pairs over each arm's busy span.  Each rate runs several arrival
    traces (Poisson at one request per second, scaled by the rate: the specs' own, then seeded
    reorderings of the same requests with fresh exponential gaps); percentiles are per trace
    and their mean is reported."""
    import queue
    import threading

    import numpy as np
    import torch

    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    from paper_2506_23809_gb300 import inputs as I
    build.build()
    B.load_library()
    torch.cuda.set_device(0)
    specs = I.serving_request_specs(args.requests, 1.0)     # arrival times at one request per second
    t_gen = time.perf_counter()
    reqs = []
    for sp in specs:
        K = sp["n_orb"] // 2
        ints = I.make_integrals(K, sp["n_orb"], sp["seed"])
        keys = I.rank_weighted_samples(K, sp["n_elec"] // 2, sp["n_elec"] // 2, sp["n_u"], seed=sp["seed"] + 1)
        reqs.append(dict(t=sp["t_arrive"], n_orb=sp["n_orb"], n_elec=sp["n_elec"], ints=ints, keys=keys,
                         counts=I.zipf_counts(sp["n_u"], 100 * sp["n_u"], sp["seed"] + 2),
                         psi=I.lognormal_psi(sp["n_u"], sp["seed"] + 3),
                         pairs=sp["n_u"] * _pairs(sp["n_orb"], sp["n_elec"])))
    t_gen = time.perf_counter() - t_gen
    n = len(reqs)
    total_pairs = sum(r["pairs"] for r in reqs)
    base_t = np.array([r["t"] for r in reqs])

    def plain_one(r):
        h = B.qc_eloc_create(r["ints"].h, r["ints"].eri, 0.0, r["n_orb"], r["n_elec"])
        e, _ = B.qc_eloc_eval(h, B.keys_to_tensor(r["keys"]), torch.from_numpy(r["counts"]).cuda(),
                              torch.from_numpy(r["psi"]).cuda())
        out = e.cpu().numpy()
        summ = B.qc_eloc_summary_read(h)
        B.qc_eloc_destroy(h)
        return out, summ

    # warm-up (kernel loading, allocator pools), then capacity: every request back to back
    plain_one(min(reqs, key=lambda r: len(r["keys"])))
    torch.cuda.synchronize()
    service = []
    for r in reqs:
        t0 = time.perf_counter()
        plain_one(r)
        service.append(time.perf_counter() - t0)
    capacity = n / sum(service)                         # requests per second, plain
    rates = [float(x) for x in args.rates.split(",")] if args.rates else \
        [0.3 * capacity, 0.7 * capacity, 1.5 * capacity]

    def plain_live(t_arr):
        q = queue.Queue()
        done = np.zeros(n)
        start = time.perf_counter()

        def client():
            for i in np.argsort(t_arr, kind="stable"):
                d = start + t_arr[i] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                q.put(int(i))
            q.put(None)
        th = threading.Thread(target=client)
        th.start()
        t_first = None
        while True:
            i = q.get()
            if i is None:
                break
            if t_first is None:
                t_first = time.perf_counter() - start
            plain_one(reqs[i])
            done[i] = time.perf_counter() - start
        th.join()
        lat = 1e3 * (done - t_arr)
        return lat, total_pairs / (done.max() - t_first), done.max()

    def served(t_arr):
        srv = B.qc_server_create(0, 160 << 30, max_slots=64, n_streams=2)
        B.qc_server_set_option(srv, B.QC_SRV_OPT_QUANTUM, int(args.quantum))
        B.qc_server_set_option(srv, B.QC_SRV_OPT_OLDEST_PCT, int(args.oldest_pct))
        if args.wave_rows >= 0:
            B.qc_server_set_option(srv, B.QC_SRV_OPT_WAVE_ROWS, int(args.wave_rows))
        res = {}
        tickets = [None] * n
        start = time.perf_counter()

        def client():
            for i in np.argsort(t_arr, kind="stable"):
                d = start + t_arr[i] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                r = reqs[i]
                tickets[i] = B.qc_eloc_submit(srv, r["ints"].h, r["ints"].eri, 0.0, r["n_orb"], r["n_elec"],
                                              r["keys"], r["counts"], r["psi"], mol_key=i + 1,
                                              borrow_integrals=True)
        th = threading.Thread(target=client)
        th.start()
        while len(res) < n:
            for i, t in enumerate(tickets):
                if t is not None and i not in res:
                    out = B.qc_eloc_poll(srv, t, 1000)
                    if out is not None:
                        res[i] = out[0]
            time.sleep(0.0005)
        th.join()
        B.qc_server_destroy(srv)
        lat = np.array([res[i]["t_done"] - res[i]["t_submit"] for i in range(n)]) * 1e3
        span = max(res[i]["t_done"] for i in range(n)) - min(res[i]["t_submit"] for i in range(n))
        stages = {k: float(np.median([1e3 * (res[i][b] - res[i][a]) for i in range(n)]))
                  for k, a, b in (("submit_to_admit", "t_submit", "t_admit"), ("admit_to_start", "t_admit", "t_start"),
                                  ("start_to_done", "t_start", "t_done"))}
        served.stages = stages
        return lat, total_pairs / span, all(res[i]["status"] == 0 for i in range(n))

    traces = [base_t]
    for k in range(1, max(1, args.serve_traces)):
        rng = np.random.default_rng(9200 + k)
        t = np.empty(n)
        t[rng.permutation(n)] = np.cumsum(rng.exponential(1.0, n))
        traces.append(t)

    def pct(x):
        return {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99)), "max": float(x.max())}

    per_rate = []
    for rate in rates:
        runs_s, runs_p, thr_s, thr_p, stages, ok = [], [], [], [], [], True
        for tb in traces:
            t_arr = tb / rate
            lp, tp_, _ = plain_live(t_arr)
            ls, ts_, ok_ = served(t_arr)
            runs_p.append(pct(lp))
            runs_s.append(pct(ls))
            thr_p.append(tp_)
            thr_s.append(ts_)
            stages.append(served.stages)
            ok = ok and ok_

        def mean(runs):
            return {k: float(np.mean([r[k] for r in runs])) for k in ("p50", "p99", "max")}
        per_rate.append({"rate_per_s": rate, "load_vs_plain_capacity": rate / capacity, "traces": len(traces),
                         "served_ms": mean(runs_s), "plain_fifo_live_ms": mean(runs_p),
                         "served_ms_per_trace": runs_s, "plain_fifo_live_ms_per_trace": runs_p,
                         "served_sustained_pairs_per_s": float(np.mean(thr_s)),
                         "plain_sustained_pairs_per_s": float(np.mean(thr_p)),
                         "served_median_stage_ms": {k: float(np.mean([s[k] for s in stages])) for k in stages[0]},
                         "all_ok": bool(ok)})
        print(json.dumps({"form": "serve", "progress": per_rate[-1]}), file=sys.stderr, flush=True)
    sat = per_rate[-1]
    line = {"metric": METRIC, "form": "serve", "value": sat["served_sustained_pairs_per_s"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f64",
            "config": {"workload": f"serve_{n}_requests_poisson_3_rates", "requests": n, "budget_gb": 160,
                       "wave_quantum_pairs": int(args.quantum), "oldest_share_pct": int(args.oldest_pct),
                       "wave_rows": int(args.wave_rows) if args.wave_rows >= 0 else 65536, "arrival_traces": len(traces),
                       "streams": 2, "n_orb_range": [min(r["n_orb"] for r in reqs), max(r["n_orb"] for r in reqs)],
                       "n_u_range": [int(min(len(r["keys"]) for r in reqs)), int(max(len(r["keys"]) for r in reqs))],
                       "samples_total": int(sum(len(r["keys"]) for r in reqs)), "pairs_total": int(total_pairs),
                       "integral_rank": "N", "input_generation_s": t_gen},
            "plain_capacity_req_per_s": capacity, "plain_back_to_back_s": float(sum(service)),
            "rates": per_rate}
    print(json.dumps(line), flush=True)
    return 0


def run_grad(args):
    """Eq. 4 gradient on the bench workload: after one evaluation, each step forms the
    weights and contracts them with n_u x P complex d ln Psi* rows (synthetic, resident in
    HBM, larger than L2).  Bound by HBM: the rows are read once, 16 B per element."""
    import numpy as np
    import torch

    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    build.build()
    B.load_library()
    torch.cuda.set_device(0)
    spec, (ints, s) = _make_workload(args.workload, 1)
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, spec["n_orb"], spec["n_elec"])
    keys = B.keys_to_tensor(s.keys)
    ct = torch.from_numpy(s.counts).cuda()
    e, _ = B.qc_eloc_eval(h, keys, ct, torch.from_numpy(s.psi).cuda())
    n_u, P = len(s.keys), int(args.n_par)
    g = torch.Generator(device="cuda").manual_seed(4401)
    D = torch.randn(n_u, P, dtype=torch.complex128, device="cuda", generator=g)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for _ in range(args.warmup):
        B.qc_eloc_grad(h, e, ct, D, weights=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in evs:
        a.record(stream)
        B.qc_eloc_grad(h, e, ct, D, weights=True)
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = t0.elapsed_time(t1)
    B.qc_eloc_destroy(h)
    peaks, peak_src = _measured_peaks()
    bytes_step = n_u * P * 16 + n_u * (16 + 8) * 2 + n_u * 16 + P * 8
    mean_s = statistics.mean(ms) / 1e3
    line = {"metric": "Eq. 4 gradient: d ln Psi* rows contracted per second", "form": "grad",
            "value": n_u * P / mean_s, "unit": "row elements/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic (Gaussian complex d ln Psi* rows, bench workload E_loc)",
            "config": {"workload": args.workload, "n_u": n_u, "n_par": P, "rows_bytes": n_u * P * 16,
                       "l2": "rows larger than L2 (read once per step)"},
            # two FP64 fused multiply-adds (4 flops) per element against the nominal FP64
            # rate of the part (no measured FP64 peak exists); HBM fraction beside it
            "roofline": {"bound": "fp64", "achieved": 4.0 * n_u * P / mean_s / 1e9, "peak": FP64_NOMINAL_GFLOPS,
                         "unit": "GFLOP/s", "frac": 4.0 * n_u * P / mean_s / 1e9 / FP64_NOMINAL_GFLOPS,
                         "traffic": None, "peak_source": "nominal FP64 rate (no measured FP64 peak)",
                         "hbm": {"achieved_gbs": bytes_step / mean_s / 1e9, "peak_gbs": peaks.get("hbm_gbs"),
                                 "frac": bytes_step / mean_s / 1e9 / peaks.get("hbm_gbs", 6800.0),
                                 "peak_source": peak_src, "algorithmic_bytes_per_step": bytes_step}},
            "gpu_launches": 3 * args.steps, "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_dedup(args):
    """The sample table built on the device from a raw stream: the bench workload's unique
    samples repeated by their counts (10^7 draws) and shuffled; each step sorts the stream
    and counts multiplicities.  The result must reproduce the sample set exactly."""
    import numpy as np
    import torch

    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    build.build()
    B.load_library()
    torch.cuda.set_device(0)
    spec, (ints, s) = _make_workload(args.workload, 1)
    rng = np.random.default_rng(4402)
    raw = np.repeat(s.keys, s.counts, axis=0)
    raw = raw[rng.permutation(raw.shape[0])]
    n = raw.shape[0]
    t_raw = torch.from_numpy(raw.view(np.int64)).cuda()
    keys = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    counts = torch.empty(n, dtype=torch.int64, device="cuda")
    nu = torch.empty(1, dtype=torch.int64, device="cuda")
    work = torch.empty(B.qc_dedup_workspace_bytes(n) + 256, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        B.qc_dedup(t_raw, spec["n_orb"], keys, counts, nu, work)
    torch.cuda.synchronize()
    ok = (int(nu.item()) == s.n_u and np.array_equal(keys[:s.n_u].cpu().numpy().view(np.uint64), s.keys)
          and np.array_equal(counts[:s.n_u].cpu().numpy(), s.counts))
    sampler = ClockSampler(0)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in evs:
        a.record(stream)
        B.qc_dedup(t_raw, spec["n_orb"], keys, counts, nu, work)
        b.record(stream)
    torch.cuda.synchronize()
    sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    peaks, peak_src = _measured_peaks()
    passes = (spec["n_orb"] + 7) // 8
    # per pass: the histogram reads each key, the scatter reads and writes it (48 B); then
    # the run pass reads the sorted keys twice (flags, emit: 32 B) and writes the table
    bytes_step = passes * 48 * n + 32 * n + 24 * s.n_u
    mean_s = statistics.mean(ms) / 1e3
    line = {"metric": "sample-table construction: raw sampled bitstrings sorted and counted per second",
            "form": "dedup", "value": n / mean_s, "unit": "raw samples/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True, "dtype": "u64",
            "data": "synthetic (the bench workload's samples repeated by their Zipf counts, shuffled)",
            "config": {"workload": args.workload, "n_raw": n, "n_unique": s.n_u, "n_orb": spec["n_orb"],
                       "radix_passes": passes, "l2": "stream (160 MB) larger than L2"},
            "exact": bool(ok),
            "roofline": {"bound": "hbm", "achieved": bytes_step / mean_s / 1e9, "peak": peaks.get("hbm_gbs"),
                         "unit": "GB/s", "frac": bytes_step / mean_s / 1e9 / peaks.get("hbm_gbs", 6800.0),
                         "traffic": None, "peak_source": peak_src, "algorithmic_bytes_per_step": bytes_step},
            "gpu_launches": (5 * passes + 6) * args.steps, "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_full(args):
    """The accurate energy at scale on a chunk of the bench workload: export the whole
    connected set (keys and elements, 24 B per pair written), then apply psi on it (24 B
    per pair read; psi here is synthetic -- in use it comes from the network)."""
    import torch

    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    build.build()
    B.load_library()
    torch.cuda.set_device(0)
    spec, (ints, s) = _make_workload(args.workload, 1)
    rows = min(int(args.chunk), s.n_u)
    h = B.qc_eloc_create(ints.h, ints.eri, 0.0, spec["n_orb"], spec["n_elec"])
    P = B.qc_eloc_pairs_per_sample(h)
    kt = B.keys_to_tensor(s.keys[:rows])
    psi = torch.from_numpy(s.psi[:rows]).cuda()
    ct = torch.from_numpy(s.counts[:rows]).cuda()
    g = torch.Generator(device="cuda").manual_seed(4403)
    pc = torch.randn(rows * P, dtype=torch.complex128, device="cuda", generator=g)
    stream = torch.cuda.current_stream()
    k = e = d = None

    def export():
        nonlocal k, e, d
        k, e, d = B.qc_eloc_export(h, kt)

    def apply():
        B.qc_eloc_apply(h, psi, ct, e, d, pc, summary=False)
    for _ in range(args.warmup):
        export()
        apply()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    t = {"export": [], "apply": []}
    for _ in range(args.steps):
        for name, fn in (("export", export), ("apply", apply)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            t[name].append(a.elapsed_time(b))
    sampler.stop()
    B.qc_eloc_destroy(h)
    peaks, peak_src = _measured_peaks()
    pairs = rows * P
    ms_e, ms_a = statistics.mean(t["export"]), statistics.mean(t["apply"])
    hbm = peaks.get("hbm_gbs", 6800.0)
    bytes_e = pairs * 24 + rows * (16 + 8)
    bytes_a = pairs * 24 + rows * (16 + 8 + 8 + 16)
    line = {"metric": "accurate energy at scale: connected pairs exported and applied per second", "form": "full",
            "value": pairs / ((ms_e + ms_a) / 1e3), "unit": "connected matrix elements/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_e + ms_a, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic (bench workload chunk; Gaussian psi on the connected set)",
            "config": {"workload": args.workload, "rows": rows, "pairs_per_sample": P, "pairs": pairs,
                       "export_bytes": bytes_e, "apply_bytes": bytes_a},
            "ms": {"export": ms_e, "apply": ms_a},
            "roofline": {"bound": "hbm", "achieved": (bytes_e + bytes_a) / ((ms_e + ms_a) / 1e3) / 1e9,
                         "peak": hbm, "unit": "GB/s", "frac": (bytes_e + bytes_a) / ((ms_e + ms_a) / 1e3) / 1e9 / hbm,
                         "traffic": None, "peak_source": peak_src,
                         "export_frac": bytes_e / (ms_e / 1e3) / 1e9 / hbm,
                         "apply_frac": bytes_a / (ms_a / 1e3) / 1e9 / hbm},
            "gpu_launches": 4 * args.steps, "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args):
    """The paper's molecular shapes (N2, PH3, LiCl of Table I; Fe2S2, H50, C6H6 of Sec. IV-B)
    with seeded synthetic integrals and rank-weighted samples: one plain step per system
    (FP64, the library's default launch), timed like the default benchmark, beside the oracle
    on the host cores over a bounded sample of rows.  One JSON line per system, then a
    summary line."""
    import numpy as np
    import torch

    import oracle
    from paper_2506_23809_gb300 import binding as B
    from paper_2506_23809_gb300 import build
    from paper_2506_23809_gb300 import inputs as I
    build.build()
    B.load_library()
    oracle.build()
    torch.cuda.set_device(0)
    prec = B.QC_FP64 if args.precision == "fp64" else B.QC_FP32_COMP
    cores = len(os.sched_getaffinity(0))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    rows_out = []
    names = [n for n, _, _ in I.PAPER_SYSTEMS] if not args.systems else args.systems.split(",")
    for name in names:
        spec, ints, s = I.paper_system_workload(name)
        h = B.qc_eloc_create(ints.h, ints.eri, 0.0, spec["n_orb"], spec["n_elec"], prec)
        B.qc_eloc_set_option(h, B.QC_OPT_TIMING, 1)
        kd = B.keys_to_tensor(s.keys)
        cd = torch.from_numpy(s.counts).cuda()
        pd = torch.from_numpy(s.psi).cuda()
        el = torch.empty(s.n_u, dtype=torch.complex128, device="cuda")
        B.qc_eloc_reserve(h, s.n_u, s.n_u)
        for _ in range(args.warmup):
            B.qc_eloc_eval(h, kd, cd, pd, eloc=el, stream=stream)
        torch.cuda.synchronize()
        ms, main = [], []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            B.qc_eloc_eval(h, kd, cd, pd, eloc=el, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            main.append(B.qc_eloc_timings(h)[1])
        summ = B.qc_eloc_summary_read(h, stream)
        cfg = B.qc_eloc_last_config(h)
        P = B.qc_eloc_pairs_per_sample(h)
        got = el.cpu().numpy()
        B.qc_eloc_destroy(h)
        step_s = statistics.mean(ms) / 1e3
        # the oracle on a bounded seeded sample of rows (each looked up in the whole table)
        rng = np.random.default_rng(spec["seed"])
        n_cpu = int(min(s.n_u, max(2 * cores, args.cpu_seconds * 3e8 / max(P, 1) / 4)))
        if args.no_cpu_baseline:
            n_cpu = 2
        sel = np.sort(rng.choice(s.n_u, n_cpu, replace=False))
        t = time.perf_counter()
        want = oracle.eloc(ints.h, ints.eri, 0.0, spec["n_orb"], s.keys[sel], s.psi[sel], s.keys, s.psi,
                           nthreads=cores)
        t_cpu = time.perf_counter() - t
        err = np.abs(got[sel] - want) / np.maximum(1.0, np.abs(want))
        line = {"metric": METRIC, "form": "sweep", "system": name, "value": s.n_u * P / step_s, "unit": UNIT,
                "samples_per_s": s.n_u / step_s, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * step_s, "main_ms": statistics.mean(main), "higher_is_better": True,
                "dtype": "f64" if prec == B.QC_FP64 else "f32+f64",
                "data": "synthetic (seeded integrals of the system's size, rank-weighted unique samples)",
                "config": {"workload": f"paper_shape_{name}", "n_orb": spec["n_orb"], "n_elec": spec["n_elec"],
                           "n_u": s.n_u, "pairs_per_sample": P, "launch": cfg,
                           "l2": "256 MB buffer written between timed steps"},
                "hits_per_step": int(summ["n_hits"]), "status": int(summ["status"]),
                "max_rel_err_vs_oracle": float(err.max()),
                "cpu_baseline": {"value": n_cpu * P / t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "samples_per_s": n_cpu / t_cpu,
                                 "sample": f"{n_cpu} seeded random rows of the {s.n_u}-row table, {t_cpu:.1f} s"}}
        rows_out.append(line)
        print(json.dumps(line), flush=True)
    print(json.dumps({"form": "sweep", "summary": [
        {"system": r["system"], "n_orb": r["config"]["n_orb"], "n_elec": r["config"]["n_elec"],
         "n_u": r["config"]["n_u"], "ms_per_step": r["ms_per_step"], "samples_per_s": r["samples_per_s"],
         "pairs_per_s": r["value"], "oracle_pairs_per_s": r["cpu_baseline"]["value"],
         "max_rel_err": r["max_rel_err_vs_oracle"]} for r in rows_out]}), flush=True)
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "batched":
        return run_batched(args)
    if args.form == "serve":
        return run_serve(args)
    if args.form == "grad":
        return run_grad(args)
    if args.form == "dedup":
        return run_dedup(args)
    if args.form == "full":
        return run_full(args)
    if args.form == "sweep":
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
