#!/usr/bin/env python
"""Benchmark of the CALU / CAQR hot path on GB300.

One step = CALU (tournament pivoting over the reduction tree) + getrs, then
CAQR (TSQR panels + tree update) + geqrs, of one n x n FP64 matrix already
resident in HBM (n = 16384, b = 128, leaves of 1024 rows).  The input is
A = U diag(s) V^T with orthogonal U, V and log-spaced s (cond 1e6) and one
right-hand side; every step restores A from a pristine device copy.

Prints one JSON line: GFLOP/s over the standard flop counts (LU 2n^3/3,
QR 4n^3/3, solves), the roofline of the dominant kernel measured live with
CUDA events on its launch stream, the oracle timed on the host cores on a
bounded sample, an end-to-end number through the public API with host
buffers, the SM clocks sampled during the timed region and the number of
library kernel launches.

--impl reference runs the CPU oracle (plain C, FP64) on the host cores on a
bounded sample of the same workload (the only other code path that may run
the oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CALU/CAQR GFLOP/s & % roofline (n=16384, FP64 vs mixed+IR); solves/s, p99 lat"
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07    # SMs x DFMA/clk/SM x flops/DFMA x max GHz = 1258.6 GFLOP/s
FP32_PEAK_DERIVED = 152 * 128 * 2 * 2.07  # SMs x FP32 lanes/SM x flops/FFMA x max GHz = 80548 GFLOP/s
# The FP64 / FP32 denominators: the FMA peak probe measured at the start of
# the run (measure_fma_peaks), the derived figures until then.
PEAKS = {"fp64": FP64_PEAK_DERIVED, "fp32": FP32_PEAK_DERIVED, "source": "derived"}
# Leaves of the n = 16384 step's tree.  Measured on GB300 (FP64 step, b = 128):
# 256 rows 747 GFLOP/s, 512 rows 844, 1024 rows 881 -- bigger leaves mean
# fewer merges, whose tree update executes more flops than the standard count.
BENCH_LEAF_ROWS = 1024


def _hbm_peak() -> float:
    """Measured copy bandwidth of this machine's GB300 (MEASURED_PEAKS.json),
    else the profiling recipe's fallback 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_GBS = _hbm_peak()


def _bf16_peaks():
    """Measured cuBLAS bf16 GEMM throughput of this machine's GB300
    (MEASURED_PEAKS.json: burst, sustained), else the profiling recipe's
    fallback 1900 / 1700 TFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 1700.0, "fallback"


BF16_TFLOPS, BF16_TFLOPS_SUSTAINED, BF16_SOURCE = _bf16_peaks()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--b", type=int, default=128)
    p.add_argument("--leaf", type=int, default=BENCH_LEAF_ROWS)
    p.add_argument("--tree", default=BENCH_TREE,
                   help="reduction-tree levels: fan-in + b (binary) or f (flat), last fan-in 0")
    p.add_argument("--cond", type=float, default=1e6)
    p.add_argument("--nrhs", type=int, default=1)
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--c3-sizes", default="4096,8192,16384")
    p.add_argument("--c3-conds", default="1e2,1e6,1e10")
    p.add_argument("--no-c3", action="store_true")
    p.add_argument("--only-c3", action="store_true", help="diagnostic: run only the n x cond grid")
    p.add_argument("--only-tslu-panel", default="",
                   help="diagnostic for profiling: M,B -- tslu of a seeded M x B panel with the benchmark's "
                        "leaves and tree, twice (the second call is the one to capture)")
    p.add_argument("--aux-steps", type=int, default=2,
                   help="timed runs of each secondary measurement (LU forms, C3 grid), after one warm-up")
    p.add_argument("--cpu-n", type=int, default=2048,
                   help="order of the oracle sample timed for cpu_baseline (about 10 s on one core)")
    p.add_argument("--ref-n", type=int, default=1024,
                   help="order of the oracle sample of each step of --impl reference (about 1 s)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--mixed-slices", type=int, default=4)
    p.add_argument("--mixed-exact", type=int, default=1)
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--serve-rates", default="100,1000,10000,100000", help="arrival rates of the sweep (requests/s)")
    p.add_argument("--serve-count", type=int, default=24, help="requests per rate (the same shapes at every rate)")
    p.add_argument("--serve-nmax", type=int, default=8192)
    p.add_argument("--serve-cond-max", type=float, default=1e8)
    p.add_argument("--serve-slots", type=int, default=4, help="concurrent requests (one stream each)")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--batch-count", type=int, default=4096, help="matrices of the batched workload")
    p.add_argument("--batch-steps", type=int, default=3)
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-configs", action="store_true")
    p.add_argument("--derive-traffic", default="",
                   help="LEAF_RATE,MERGE_RATE: DRAM bytes per C element of a wide leaf / merge launch "
                        "(ncu); prints the per-launch traffic line for this workload and exits (no GPU)")
    p.add_argument("--only-serve", action="store_true", help="diagnostic: run only the serving workload")
    p.add_argument("--only-configs", action="store_true", help="diagnostic: run only the other configurations")
    p.add_argument("--only-batch", default="", choices=["", "f64", "f32", "ops"],
                   help="diagnostic: run only the batched workload in this precision")
    return p.parse_args()


def step_flops(n: int, nrhs: int) -> float:
    lu = 2.0 * n ** 3 / 3.0
    qr = 4.0 * n ** 3 / 3.0
    getrs = 2.0 * n * n * nrhs
    geqrs = 3.0 * n * n * nrhs
    return lu + qr + getrs + geqrs


BENCH_TREE = "4f,0f"  # one flat merge per group of 4 leaves, then one flat merge of the groups


def parse_tree(spec: str):
    """Reduction-tree levels from "f<style>,..." (fan-in, b = binary merges,
    f = one flat merge of the group; fan-in 0 = all remaining nodes)."""
    out = []
    for tok in spec.split(","):
        tok = tok.strip()
        if not tok or tok[-1] not in "bf" or not tok[:-1].isdigit():
            raise ValueError(f"bad tree level {tok!r} (want e.g. 4b or 0f)")
        out.append((int(tok[:-1]), 0 if tok[-1] == "b" else 1))
    if out[-1][0] != 0:
        raise ValueError("the last tree level must have fan-in 0 (all remaining nodes)")
    return out


def describe_tree(levels) -> str:
    words = []
    for f, st in levels:
        kind = "binary" if st == 0 else "flat"
        words.append(f"{kind} merges over {'all remaining nodes' if f == 0 else f'groups of {f}'}")
    return ", then ".join(words)


def workload_config(a, extra=None):
    c = {
        "workload": (f"CALU+getrs and CAQR+geqrs of one {a.n}x{a.n} FP64 matrix "
                     f"(A = U diag(s) V^T, cond {a.cond:g}), b={a.b}, leaves of {a.leaf} rows, "
                     f"reduction tree {a.tree}, {a.nrhs} RHS"),
        "n": a.n, "b": a.b, "leaf_rows": a.leaf, "tree": describe_tree(parse_tree(a.tree)),
        "cond": a.cond, "nrhs": a.nrhs, "precision": "plain FP64",
        "l2": "inputs (8 n^2 bytes) larger than the 129 MB L2",
    }
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
REJECT_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clocks) -> bool:
    """Whether a timed region's clock record disqualifies it: a hardware or
    thermal slowdown was active, or the SM clock sat well below its maximum
    with no reason active (a clock left locked).  sw_power_cap alone is kept
    (and noted in the record)."""
    if not clocks or clocks.get("sm_mhz") is None or not clocks.get("sm_max_mhz"):
        return False
    reasons = clocks.get("reasons") or []
    if any(r in REJECT_REASONS for r in reasons):
        return True
    return not reasons and clocks["sm_mhz"] < 0.85 * clocks["sm_max_mhz"]


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(a, n: int):
    """CALU + getrs and CAQR + geqrs by the CPU oracle on an n x n matrix of
    the same family; returns (seconds, flops)."""
    import oracle
    from paper_1303_5837_gb300 import inputs
    A = inputs.conditioned(n, a.cond, 2026)
    B = inputs.rhs(n, a.nrhs, 2027)
    tree = oracle.make_tree(a.leaf, parse_tree(a.tree))
    oracle.build()
    t0 = time.perf_counter()
    LU, ipiv, _, _ = oracle.calu(A, a.b, tree)
    oracle.getrs(LU, ipiv, B)
    QR, T = oracle.caqr(A, a.b, tree)
    oracle.geqrs(QR, T, a.b, tree, B)
    return time.perf_counter() - t0, step_flops(n, a.nrhs)


def _oracle_worker(job, barrier, out):
    """One oracle sample in a spawned process: every worker starts its timed
    computation at the same barrier, then reports (start, end, flops)."""
    cond, nrhs, b, leaf, tree, n = job
    import oracle
    from paper_1303_5837_gb300 import inputs
    A = inputs.conditioned(n, cond, 2026)
    B = inputs.rhs(n, nrhs, 2027)
    t = oracle.make_tree(leaf, parse_tree(tree))
    try:
        barrier.wait(timeout=300)
    except threading.BrokenBarrierError:
        pass
    t0 = time.monotonic()
    LU, ipiv, _, _ = oracle.calu(A, b, t)
    oracle.getrs(LU, ipiv, B)
    QR, T = oracle.caqr(A, b, t)
    oracle.geqrs(QR, T, b, t, B)
    out.put((t0, time.monotonic(), step_flops(n, nrhs)))


def usable_cores():
    """(cores this process may run on, where the figure came from): the CPU
    affinity mask (which honours cgroup / container limits set through it),
    else os.cpu_count()."""
    try:
        return len(os.sched_getaffinity(0)), "sched_getaffinity"
    except (AttributeError, OSError):
        return os.cpu_count() or 1, "os.cpu_count"


def cpu_baseline_all_cores(a, cores=None):
    """The same oracle (unchanged, single-threaded) on every host core at
    once: one process per core, each on its own copy of the sample matrix,
    started together; aggregate flops over the span from the first start to
    the last end.  Processes are spawned (never forked from a process that
    holds a CUDA context)."""
    import multiprocessing as mp
    import queue as _queue
    import oracle
    oracle.build()
    cores_source = "argument"
    if not cores:
        cores, cores_source = usable_cores()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    out = ctx.Queue()
    job = (a.cond, a.nrhs, a.b, a.leaf, a.tree, a.cpu_n)
    procs = [ctx.Process(target=_oracle_worker, args=(job, barrier, out), daemon=True) for _ in range(cores)]
    # one BLAS thread per worker (the inputs are generated with numpy; the
    # oracle itself is plain C): the children inherit the environment
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in saved})
    try:
        for p in procs:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    res = []
    deadline = time.monotonic() + 900
    while len(res) < cores and time.monotonic() < deadline:
        try:
            res.append(out.get(timeout=1.0))
        except _queue.Empty:
            # a worker that died without a result ends the measurement
            if any(p.exitcode not in (None, 0) for p in procs) or not any(p.is_alive() for p in procs):
                if out.empty():
                    break
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    if len(res) != cores:
        return None
    span = max(r[1] for r in res) - min(r[0] for r in res)
    flops = sum(r[2] for r in res)
    return {"value": flops / span / 1e9, "unit": "GFLOP/s", "cores": cores, "cores_source": cores_source,
            "kind": "oracle",
            "sample": (f"{cores} concurrent copies (one process per host core) of the single-core sample: "
                       f"oracle CALU+getrs and CAQR+geqrs of one {a.cpu_n}x{a.cpu_n} matrix each, "
                       f"{span:.1f} s"),
            "seconds": span}


def cpu_baseline(a):
    secs, fl = oracle_sample(a, a.cpu_n)
    return {"value": fl / secs / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle CALU+getrs and CAQR+geqrs of one {a.cpu_n}x{a.cpu_n} matrix of the "
                       f"same family (b={a.b}, leaves {a.leaf}), single-threaded C, {secs:.1f} s"),
            "seconds": secs}


def run_reference(a, rank: int, world: int):
    if rank != 0:
        return
    times = []
    for i in range(a.warmup + a.steps):
        secs, fl = oracle_sample(a, a.ref_n)
        if i >= a.warmup:
            times.append(secs)
    t = sum(times)
    value = fl * len(times) / t / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * t / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": workload_config(a, {"sample_n": a.ref_n}),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: oracle on one {a.ref_n}x{a.ref_n} matrix"},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def tree_rounds(nleaves: int, levels):
    """Merge rounds of the reduction tree over `nleaves` leaves, as the
    library plans them (one launch per round): per round, the number of
    inputs of each output node, in order.  Per level, groups of fan_in
    consecutive nodes (the last level takes all); binary style pairs
    neighbours until one node is left per group (an odd one passes through),
    flat style merges a group at once.  Rounds without a merge are dropped."""
    rounds = []
    cur = nleaves
    for li, (fan, style) in enumerate(levels):
        f = cur if li == len(levels) - 1 else fan
        ngroups = -(-cur // f)
        sizes = [f] * (ngroups - 1) + [cur - (ngroups - 1) * f] if ngroups > 1 else [cur]
        if style == 1:
            if any(g >= 2 for g in sizes):
                rounds.append(list(sizes))
        else:
            while any(g > 1 for g in sizes):
                rnd, nxt = [], []
                for g in sizes:
                    outs = [2] * (g // 2) + ([1] if g % 2 else [])
                    rnd += outs
                    nxt.append(len(outs))
                rounds.append(rnd)
                sizes = nxt
        cur = ngroups
    return rounds


def tree_update_launches(n: int, b: int, leaf: int, levels, nrhs: int, sms: int = 152):
    """The tree-update launches of one benchmark step (caqr_factor with the
    look-ahead, then caqr_geqrs), in order: (kernel, is_leaf, C elements).
    The library runs an update on the narrow kernel when it has at most 8
    columns or its leaf launch would have fewer 32-column CTAs than SMs.
    C elements: a leaf launch touches every panel row of its columns, a
    merge launch the stacked R rows of the nodes that merge."""
    out = []

    def apply(mk, bk, nl, rounds, ncols):
        if ncols <= 0:
            return
        narrow = ncols <= 8 or nl * (-(-ncols // 32)) < sms
        kind = "tree_narrow" if narrow else "tree_apply"
        out.append((kind, True, mk * ncols))
        rows = [min(leaf, mk - j * leaf, bk) for j in range(nl)]   # R rows per node
        for rnd in rounds:
            nxt, at, el = [], 0, 0
            for cnt in rnd:
                kids = rows[at:at + cnt]
                at += cnt
                if cnt >= 2:
                    el += sum(kids)
                nxt.append(min(sum(kids), bk) if cnt >= 2 else kids[0])
            rows = nxt
            out.append((kind, False, el * ncols))

    panels = [(kb, min(b, n - kb)) for kb in range(0, n, b)]
    for kb, bk in panels:
        mk = n - kb
        nl = -(-mk // leaf)
        rounds = tree_rounds(nl, levels)
        nt = n - kb - bk
        if nt > 0:
            nnext = min(nt, b)
            if n > b and nnext < nt:
                apply(mk, bk, nl, rounds, nnext)
                apply(mk, bk, nl, rounds, nt - nnext)
            else:
                apply(mk, bk, nl, rounds, nt)
    for kb, bk in panels:
        mk = n - kb
        nl = -(-mk // leaf)
        apply(mk, bk, nl, tree_rounds(nl, levels), nrhs)
    return out


def derive_traffic(leaf_rate: float, merge_rate: float, n: int, b: int, leaf: int, levels,
                   nrhs: int = 1, sms: int = 152):
    """Per-launch DRAM bytes of the wide tree update over one step: DRAM
    bytes per C element of a leaf launch and per stacked C element of a merge
    launch (from an ncu capture of a smaller case) times the elements each
    wide launch processes, averaged over the wide launches."""
    ls = tree_update_launches(n, b, leaf, levels, nrhs, sms)
    wide = [(is_leaf, el) for kind, is_leaf, el in ls if kind == "tree_apply"]
    narrow = sum(1 for kind, _, _ in ls if kind == "tree_narrow")
    total = sum((leaf_rate if is_leaf else merge_rate) * el for is_leaf, el in wide)
    return {"wide_launches": len(wide), "narrow_launches": narrow,
            "bytes_per_wide_launch": total / max(1, len(wide))}


TRAFFIC_SOURCES = {"tree_apply": "panel_qr.cu#tree_apply_kernel,ca_internal.cuh#tree_plan"}


def print_traffic_line(a):
    """The profiles/traffic.txt line of the wide tree update for this
    workload, from the per-element DRAM rates of an ncu capture."""
    leaf_rate, merge_rate = (float(x) for x in a.derive_traffic.split(","))
    d = derive_traffic(leaf_rate, merge_rate, a.n, a.b, a.leaf, parse_tree(a.tree), a.nrhs)
    csrc = os.path.join(ROOT, "paper_1303_5837_gb300", "csrc")
    h = hashlib.sha256()
    for item in TRAFFIC_SOURCES["tree_apply"].split(","):
        h.update(source_text(csrc, item))
    print(f"tree_apply {TRAFFIC_SOURCES['tree_apply']} {h.hexdigest()[:16]} "
          f"{d['bytes_per_wide_launch']:.4e} plan={a.n}/{a.b}/{a.leaf}/{a.tree}/{d['wide_launches']} "
          f"per-launch average of the {d['wide_launches']} wide launches of one step "
          f"(CALU+getrs and CAQR+geqrs, n={a.n}, b={a.b}, {a.leaf}-row leaves, tree {a.tree}, "
          f"{a.nrhs} RHS; {d['narrow_launches']} narrow launches), derived by "
          f"python bench.py --derive-traffic {a.derive_traffic}: {leaf_rate} DRAM bytes per C element "
          f"of a leaf launch, {merge_rate} per stacked C element of a merge launch "
          f"(from an ncu capture of the leaf and merge launches at n=6144)")


def source_text(csrc: str, item: str) -> bytes:
    """Bytes of one source item of profiles/traffic.txt: a whole file
    ("panel_qr.cu") or the lines between "// @region NAME" and
    "// @endregion NAME" of a file ("panel_qr.cu#NAME")."""
    fname, _, region = item.partition("#")
    with open(os.path.join(csrc, fname), "rb") as fh:
        data = fh.read()
    if not region:
        return data
    begin = f"// @region {region}\n".encode()
    end = f"// @endregion {region}".encode()
    i = data.find(begin)
    j = data.find(end, i + len(begin)) if i >= 0 else -1
    if i < 0 or j < 0:
        return b""
    return data[i + len(begin):j]


def traffic_for(kernel: str, plan: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary
    (profiles/traffic.txt: kernel, its source items, a hash of them, bytes,
    plan=n/b/leaf_rows/tree/launches per step), if the counters were taken on
    the current code of that kernel and the per-launch figure was derived for
    this run's plan of launches."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    csrc = os.path.join(ROOT, "paper_1303_5837_gb300", "csrc")
    for ln in open(path):
        p = ln.split()
        if len(p) < 5 or p[0] != kernel or not p[4].startswith("plan="):
            continue
        h = hashlib.sha256()
        for item in p[1].split(","):
            h.update(source_text(csrc, item))
        if h.hexdigest()[:16] == p[2] and p[4][len("plan="):] == plan:
            return float(p[3])
    return None


def _load_torch_linalg():
    """torch loads its CUDA linear-algebra library by name on the first QR;
    under a profiler that intercepts dlopen the name is not found, so load it
    by its path first (a no-op once loaded)."""
    import ctypes
    import torch
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)


def haar_device(n, seed, dev):
    """A Haar-distributed orthogonal n x n matrix on the device: Q of the QR
    of a seeded N(0, 1) matrix with the signs of R's diagonal folded in
    (input generation, untimed; torch's QR)."""
    import torch
    _load_torch_linalg()
    g = torch.Generator(device=dev).manual_seed(seed)
    Z = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    Q, R = torch.linalg.qr(Z)
    Q *= torch.sign(torch.diagonal(R))[None, :]
    return Q


def c3_grid(a, ca, torch, dev, world):
    """Square CALU solves over the grid n x cond (b = 128, the benchmark's
    leaves and tree, one right-hand side): plain FP64 (calu_factor +
    calu_getrs) against the mixed form (calu_gesv_mixed: a.mixed_slices
    digits on the tensor cores, refinement "auto" to backward error 1e-14);
    each one warm-up and a.aux_steps timed runs.  A = U diag(s) V^T with
    s_i = cond^(-i/(n-1)); U, V Haar (QR of a seeded Gaussian), drawn once
    per n."""
    from paper_1303_5837_gb300 import inputs
    st = torch.cuda.current_stream()
    b, S = a.b, a.mixed_slices
    tree = ca.make_tree(a.leaf, parse_tree(a.tree))
    sizes = [int(x) for x in a.c3_sizes.split(",") if x]
    conds = [float(x) for x in a.c3_conds.split(",") if x]
    out = {"slices": S, "refine": "auto", "tol": 1e-14, "cells": []}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = max(1, a.aux_steps)
        e0.record(st)
        r = None
        for _ in range(reps):
            r = fn()
        e1.record(st)
        e1.synchronize()
        return allreduce_max(e0.elapsed_time(e1), world) / reps, r

    for n in sizes:
        lu_flops = 2.0 * n ** 3 / 3.0 + 2.0 * n * n
        U, V = haar_device(n, 31 + n, dev), haar_device(n, 37 + n, dev)
        family = "Haar U, V (QR of a Gaussian)"
        A = torch.empty((n, n), dtype=torch.float64, device=dev).t()
        LU = torch.empty_like(A)
        X = torch.empty((n, 1), dtype=torch.float64, device=dev)
        ipiv = torch.empty(n, dtype=torch.int32, device=dev)
        info = torch.zeros(2, dtype=torch.int32, device=dev)
        work = torch.empty((ca.ca_calu_workspace(n, n, b, tree) + 7) // 8, dtype=torch.float64, device=dev)
        swork = torch.empty((ca.ca_getrs_workspace(n, 1) + 7) // 8, dtype=torch.float64, device=dev)
        wmix = torch.empty((ca.ca_gesv_mixed_workspace(n, 1, b, tree, S, True, "auto") + 7) // 8,
                           dtype=torch.float64, device=dev)
        for cond in conds:
            s_ = torch.from_numpy(inputs.singular_values(n, cond)).to(dev)
            A0 = ((U * s_) @ V.t()).t().contiguous().t()
            x_true = torch.randn(n, 1, dtype=torch.float64, device=dev,
                                 generator=torch.Generator(device=dev).manual_seed(5))
            B0 = A0 @ x_true
            anorm = float(A0.abs().sum(1).amax())

            def berr_of(Xs):
                R = B0 - A0 @ Xs
                return float(R.abs().amax() / (anorm * Xs.abs().amax() + B0.abs().amax()))

            def plain():
                A.copy_(A0)
                X.copy_(B0)
                ca.calu_factor(A, b, tree, ipiv=ipiv, work=work, dev_info=info)
                ca.calu_getrs(A, ipiv, X, work=swork)

            ms_p, _ = timed(plain)
            be_p = berr_of(X)
            info_p = info.cpu().tolist()

            def mixed():
                return ca.calu_gesv_mixed(A0, B0, b, tree, slices=S, exact=True, max_iter=10, tol=1e-14,
                                          refine="auto", LU=LU, X=X, ipiv=ipiv, work=wmix, dev_info=info)

            ms_m, (_, it, be, inf) = timed(mixed)
            be_m, it_m, inf_m = float(be.item()), int(it.item()), inf.cpu().tolist()
            cell = {"n": n, "cond": cond, "family": family,
                    "fp64": {"ms": ms_p, "gflops": lu_flops / ms_p / 1e6, "berr": be_p, "info": info_p},
                    "mixed": {"ms": ms_m, "gflops": lu_flops / ms_m / 1e6, "berr": float(be_m),
                              "berr_check": berr_of(X), "iters": it_m, "info": inf_m,
                              "refactored": bool(inf_m[1] & ca.CA_STATUS_REFACTORED),
                              "reaches_tol": be_m <= 1e-14},
                    "speedup": ms_p / ms_m}
            out["cells"].append(cell)
            del A0, B0
        del U, V, A, LU, X, work, wmix
        torch.cuda.empty_cache()
    return out


def measure_fma_peaks(ca, torch, dev, reps: int = 5) -> dict:
    """FP64 and FP32 FMA throughput of this GPU from the library's peak probe
    (8 independent fused multiply-adds per thread per round, 8 CTAs of 256
    threads per SM), best of `reps` launches timed with CUDA events; sets
    PEAKS, the denominators of the roofline fractions."""
    out = {}
    st = torch.cuda.current_stream()
    for name, dt, tdt, iters in (("fp64", 0, torch.float64, 4000), ("fp32", 1, torch.float32, 100000)):
        blocks = 152 * 8
        buf = torch.empty(blocks * 256, dtype=tdt, device=dev)
        ca.ca_peak_probe(dt, blocks, iters, buf)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ca.ca_peak_probe(dt, blocks, iters, buf)
            e1.record(st)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        flops = 16.0 * iters * blocks * 256
        out[name] = {"gflops": flops / (best / 1e3) / 1e9, "ms": best,
                     "derived": FP64_PEAK_DERIVED if name == "fp64" else FP32_PEAK_DERIVED}
        PEAKS[name] = out[name]["gflops"]
    PEAKS["source"] = "measured (ca_peak_probe)"
    return out


def run_ours(a, rank: int, world: int, local: int):
    import torch
    import paper_1303_5837_gb300 as ca
    from paper_1303_5837_gb300 import inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ca.load()
    if a.only_tslu_panel:
        m, bw = (int(x) for x in a.only_tslu_panel.split(","))
        t = ca.make_tree(a.leaf, parse_tree(a.tree))
        P0 = torch.randn(bw, m, dtype=torch.float64, device=dev,
                         generator=torch.Generator(device=dev).manual_seed(3)).t()
        for _ in range(2):
            P = P0.t().contiguous().t()
            _, info = ca.tslu(P, t)
        torch.cuda.synchronize()
        print(json.dumps({"tslu_panel": [m, bw], "info": info.cpu().tolist()}), flush=True)
        return
    peaks = measure_fma_peaks(ca, torch, dev)
    if a.only_c3:
        res = c3_grid(a, ca, torch, dev, world)
        if rank == 0:
            print(json.dumps({"c3_grid": res, "fma_peaks": peaks}), flush=True)
        return
    if a.only_serve:
        if rank == 0:
            print(json.dumps({"serving": serving_run(a)}), flush=True)
        return
    if a.only_configs:
        if rank == 0:
            print(json.dumps({"other_configs": other_configs(a, ca, torch, dev)}), flush=True)
        return
    if a.only_batch:
        if a.only_batch == "ops":
            print(json.dumps({"batched": {"operators": operator_diagnostics(a, ca, torch, dev),
                                          "operators_8192": operator_diagnostics_large(a, ca, torch, dev)}}),
                  flush=True)
            return
        out = batched_run(a, ca, torch, torch.float64 if a.only_batch == "f64" else torch.float32, dev, rank,
                          world)
        if rank == 0:
            print(json.dumps({"batched": {a.only_batch: out}}), flush=True)
        return
    n, b, nrhs = a.n, a.b, a.nrhs
    tree = ca.make_tree(a.leaf, parse_tree(a.tree))

    # ---- inputs (untimed): A = U diag(s) V^T, B = A x_true ------------------
    A0 = conditioned_device(n, a.cond, 2026 + rank, dev)
    x_true = torch.randn(n, nrhs, dtype=torch.float64, device=dev,
                         generator=torch.Generator(device=dev).manual_seed(7 + rank))
    B0 = ca.colmajor(A0 @ x_true)
    A = torch.empty_like(A0)
    X = torch.empty_like(B0)
    ipiv = torch.empty(n, dtype=torch.int32, device=dev)
    info = torch.zeros(2, dtype=torch.int32, device=dev)
    qinfo = torch.zeros(2, dtype=torch.int32, device=dev)
    lwork = ca.ca_calu_workspace(n, n, b, tree)
    work = torch.empty((lwork + 7) // 8, dtype=torch.float64, device=dev)
    swork = torch.empty((ca.ca_getrs_workspace(n, nrhs) + 7) // 8, dtype=torch.float64, device=dev)
    qb, qw = ca.ca_caqr_workspace(n, n, b, tree)
    qtree = torch.empty((qb + 7) // 8, dtype=torch.float64, device=dev)
    qwork = torch.empty((max(qw, ca.ca_geqrs_workspace(n, n, nrhs, b, tree)) + 7) // 8,
                        dtype=torch.float64, device=dev)

    def factor_and_solve(src_A, src_B):
        A.copy_(src_A)
        X.copy_(src_B)
        ca.calu_factor(A, b, tree, ipiv=ipiv, work=work, dev_info=info)
        ca.calu_getrs(A, ipiv, X, work=swork)
        x_lu = X.clone() if check else None
        A.copy_(src_A)
        X.copy_(src_B)
        ca.caqr_factor(A, b, tree, qtree=qtree, work=qwork, dev_info=qinfo)
        ca.caqr_geqrs(A, b, tree, qtree, X, work=qwork)
        return x_lu

    def library_status():
        """What the library reported about the last step: dev_info of the
        factorizations and whether a triangular solve gave up waiting."""
        return {"calu_info": info.cpu().tolist(), "caqr_info": qinfo.cpu().tolist(),
                "getrs_timed_out": ca.ca_solve_status(swork), "geqrs_timed_out": ca.ca_solve_status(qwork)}

    def status_ok(stt):
        return (stt["calu_info"] == [0, 0] and stt["caqr_info"] == [0, 0] and not stt["getrs_timed_out"]
                and not stt["geqrs_timed_out"])

    # ---- correctness of the timed configuration (untimed) -----------------
    check = True
    x_lu = factor_and_solve(A0, B0)
    torch.cuda.synchronize()
    err_lu = float(torch.linalg.norm(x_lu - x_true) / torch.linalg.norm(x_true))
    err_qr = float(torch.linalg.norm(X - x_true) / torch.linalg.norm(x_true))
    check = False

    for _ in range(a.warmup):
        factor_and_solve(A0, B0)
    torch.cuda.synchronize()
    barrier(world)

    def timed_region():
        sampler = ClockSampler(local)
        sampler.start()
        ca.ca_prof_enable(True, 12000 * max(1, a.steps))
        launches0 = ca.ca_launch_count()
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(a.steps):
            factor_and_solve(A0, B0)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = ca.ca_launch_count() - launches0
        clocks = sampler.stop()
        kernels = {}
        for c, name in enumerate(ca.KERNEL_CLASSES):
            cnt, kms, kfl, dropped = ca.ca_prof_read(c)
            if cnt:
                kernels[name] = {"launches": cnt, "ms": kms, "gflop": kfl / 1e9, "dropped": dropped}
        ca.ca_prof_enable(False, 1)
        return ms, launches, clocks, kernels

    ms, launches, clocks, kernels = timed_region()
    lib_status = library_status()   # the last timed step's own report (a failure voids the number)
    st = torch.cuda.current_stream()
    first_clocks = None
    # a region that saw a slowdown (on any rank) is measured once more
    if allreduce_max(1.0 if clocks_rejected(clocks) else 0.0, world) > 0:
        first_clocks = clocks
        barrier(world)
        ms, launches, clocks, kernels = timed_region()
        lib_status = library_status()
    ms_max = allreduce_max(ms, world)

    flops = step_flops(n, nrhs)
    value = world * flops * a.steps / (ms_max / 1e3) / 1e9
    # dominant kernel by device time
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    dk = kernels[dom]
    achieved = dk["gflop"] / (dk["ms"] / 1e3)
    tot_kms = sum(v["ms"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = v["ms"] / tot_kms

    # ---- LU alone: plain FP64 vs mixed + refinement vs 7-digit emulation ----
    lu_forms = None
    if not a.no_mixed:
        lu_forms = lu_form_timings(a, ca, torch, A0, B0, x_true, tree, st, world)

    # ---- the n x cond grid: FP64 against mixed + refinement ----------------
    c3 = None
    if not a.no_c3:
        c3 = c3_grid(a, ca, torch, dev, world)

    # ---- serving: continuous batching of an open-loop Poisson stream ---------
    serving = None
    if not a.no_serve and world == 1:
        serving = serving_run(a)

    # ---- batched: many uneven matrices in one persistent graph-captured launch
    batched = None
    if not a.no_batch:
        batched = {}
        for tname, tdt in (("f64", torch.float64), ("f32", torch.float32)):
            batched[tname] = batched_run(a, ca, torch, tdt, dev, rank, world)
        if rank == 0:
            batched["operators"] = operator_diagnostics(a, ca, torch, dev)
            batched["operators_8192"] = operator_diagnostics_large(a, ca, torch, dev)

    # ---- the other configurations (tall-skinny panels, the small square) ----
    configs = None
    if not a.no_configs and rank == 0:
        configs = other_configs(a, ca, torch, dev)

    # ---- end to end through the public API with host buffers --------------
    e2e = None
    if a.e2e_steps > 0:
        # pinned host copies in the device tensors' own column-major layout;
        # every transfer goes through the transposed (contiguous) views, so it
        # is one contiguous copy of the whole buffer
        A_h = torch.empty(A0.shape[::-1], dtype=torch.float64).pin_memory().t()
        A_h.t().copy_(A0.t().cpu())
        B_h = torch.empty(B0.shape[::-1], dtype=torch.float64).pin_memory().t()
        B_h.t().copy_(B0.t().cpu())
        X_h = torch.empty(B0.shape[::-1], dtype=torch.float64).pin_memory().t()

        def xfer(dst, src):
            dst.t().copy_(src.t(), non_blocking=True)

        def e2e_step():
            xfer(A, A_h)                         # H2D: the matrix
            xfer(X, B_h)                         # H2D: the right-hand side
            ca.calu_factor(A, b, tree, ipiv=ipiv, work=work, dev_info=info)
            ca.calu_getrs(A, ipiv, X, work=swork)
            xfer(X_h, X)                         # D2H: the LU solution
            xfer(A, A_h)
            xfer(X, B_h)
            ca.caqr_factor(A, b, tree, qtree=qtree, work=qwork, dev_info=info)
            ca.caqr_geqrs(A, b, tree, qtree, X, work=qwork)
            xfer(X_h, X)                         # D2H: the least-squares solution

        e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(st)
        for _ in range(a.e2e_steps):
            e2e_step()
        f1.record(st)
        torch.cuda.synchronize()
        ems = allreduce_max(f0.elapsed_time(f1), world)
        h2d = 2 * A0.numel() * 8 + 2 * B0.numel() * 8
        d2h = 2 * B0.numel() * 8
        e2e = {"value": world * flops * a.e2e_steps / (ems / 1e3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": ems / a.e2e_steps}

    if rank != 0:
        return
    cpu = cpu_all = None
    if world == 1 and not a.no_cpu:
        cpu = cpu_baseline(a)
        try:  # context only: a failure here must not cost the measurement
            cpu_all = cpu_baseline_all_cores(a)
        except Exception as e:  # noqa: BLE001
            cpu_all = {"error": repr(e)}
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(a, {"parallelism": f"replicas{world}" if world > 1 else "single"}),
        "roofline": {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": PEAKS["fp64"],
                     "unit": "GFLOP/s", "frac": achieved / PEAKS["fp64"],
                     "peak_derived": FP64_PEAK_DERIVED, "frac_of_derived": achieved / FP64_PEAK_DERIVED,
                     "traffic": traffic_for(dom, f"{n}/{b}/{a.leaf}/{a.tree}/"
                                                 f"{round(dk['launches'] / a.steps)}"),
                     "peak_source": ("FP64 DFMA peak measured in this run by ca_peak_probe (8 independent "
                                     "DFMA chains per thread, 8 CTAs per SM, best of 5); derived: 152 SMs x "
                                     "2 DFMA/clk x 2 flop x 2.07 GHz")},
        "fma_peaks": peaks,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "e2e": e2e,
        "clocks": clocks if first_clocks is None else dict(clocks, remeasured_after=first_clocks),
        "gpu_launches": launches,
        "kernels": kernels,
        "check": {"x_rel_err_calu": err_lu, "x_rel_err_caqr": err_qr, "library_status": lib_status,
                  "ok": status_ok(lib_status)},
        "lu_forms": lu_forms,
        "c3_grid": c3,
        "serving": serving,
        "batched": batched,
        "other_configs": configs,
    }
    print(json.dumps(line), flush=True)


def lu_form_timings(a, ca, torch, A0, B0, x_true, tree, st, world):
    """CALU solve of A x = b three ways, each timed over a.aux_steps runs after
    one warm-up: plain FP64 (calu_factor + calu_getrs), the reduced-precision
    update on the tensor cores with FP64 refinement (calu_gesv_mixed), and the
    exact 7-digit tensor-core update (FP64-accurate factors) + calu_getrs."""
    n, b = a.n, a.b
    lu_flops = 2.0 * n ** 3 / 3.0 + 2.0 * n * n * a.nrhs
    A = torch.empty_like(A0)
    X = torch.empty_like(B0)
    ipiv = torch.empty(n, dtype=torch.int32, device=A0.device)
    info = torch.zeros(2, dtype=torch.int32, device=A0.device)
    out = {}

    kernels_of = {}

    def timed(fn, name=None):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if name:
            ca.ca_prof_enable(True, 200000)
        reps = max(1, a.aux_steps)
        e0.record(st)
        res = None
        for _ in range(reps):
            res = fn()
        e1.record(st)
        torch.cuda.synchronize()
        if name:
            ks = {}
            for c, kn in enumerate(ca.KERNEL_CLASSES):
                cnt, kms, kfl, _ = ca.ca_prof_read(c)
                if cnt:
                    ks[kn] = {"launches": cnt // reps, "ms": kms / reps, "gflop": kfl / reps / 1e9}
            ca.ca_prof_enable(False, 1)
            kernels_of[name] = ks
        return allreduce_max(e0.elapsed_time(e1), world) / reps, res

    def berr_of(Xs):
        R = B0 - A0 @ Xs
        num = R.abs().amax(0)
        den = A0.abs().sum(1).amax() * Xs.abs().amax(0) + B0.abs().amax(0)
        return float((num / den).max())

    work = torch.empty((ca.ca_calu_workspace(n, n, b, tree) + 7) // 8, dtype=torch.float64, device=A0.device)
    swork = torch.empty((ca.ca_getrs_workspace(n, a.nrhs) + 7) // 8, dtype=torch.float64, device=A0.device)

    def plain():
        A.copy_(A0)
        X.copy_(B0)
        ca.calu_factor(A, b, tree, ipiv=ipiv, work=work, dev_info=info)
        ca.calu_getrs(A, ipiv, X, work=swork)

    ms, _ = timed(plain)
    out["fp64"] = {"ms": ms, "gflops": lu_flops / ms / 1e6, "berr": berr_of(X),
                   "form": "calu_factor + calu_getrs, FP64 DFMA update"}
    S, ex = a.mixed_slices, bool(a.mixed_exact)
    LU = torch.empty_like(A0)
    wmix = torch.empty((ca.ca_gesv_mixed_workspace(n, a.nrhs, b, tree, S, ex, "auto") + 7) // 8,
                       dtype=torch.float64, device=A0.device)

    def mixed():
        _, it, be, _ = ca.calu_gesv_mixed(A0, B0, b, tree, slices=S, exact=ex, max_iter=30, tol=1e-14,
                                          refine="auto", LU=LU, X=X, ipiv=ipiv, work=wmix, dev_info=info)
        return it, be

    ms, (it, be) = timed(mixed, "mixed_ir")
    it, be = int(it.item()), float(be.item())
    mixed_ms = ms
    out["mixed_ir"] = {"ms": ms, "gflops": lu_flops / ms / 1e6, "iters": it, "berr": be, "refine": "auto",
                       "berr_check": berr_of(X), "slices": S, "exact": ex,
                       "x_rel_err": float(torch.linalg.norm(X - x_true) / torch.linalg.norm(x_true)),
                       "speedup_vs_fp64": out["fp64"]["ms"] / ms,
                       "form": f"calu_gesv_mixed: {S}-digit bf16 tensor-core update + FP64 refinement",
                       "kernels_note": ("launch records of every kernel enqueued, including the phases that the "
                                        "device skips once refinement has converged (the GMRES and the 7-digit "
                                        "refactorization phases of refine=auto): those launches return at once, "
                                        "and their flop figures were not executed; mixed_factor below holds the "
                                        "factorization alone")}
    wfac = torch.empty((ca.ca_calu_mixed_workspace(n, n, b, tree, S, ex) + 7) // 8, dtype=torch.float64,
                       device=A0.device)

    def mixed_factor():
        A.copy_(A0)
        ca.calu_factor_mixed(A, b, tree, slices=S, exact=ex, ipiv=ipiv, work=wfac, dev_info=info)

    ms, _ = timed(mixed_factor, "mixed_factor")
    out["mixed_factor"] = {"ms": ms, "gflops": 2.0 * n ** 3 / 3.0 / ms / 1e6,
                           "share_of_mixed_ir": ms / mixed_ms,
                           "form": f"calu_factor_mixed({S} digits), the factorization of mixed_ir alone"}
    del wfac
    wemu = torch.empty((ca.ca_calu_mixed_workspace(n, n, b, tree, 7, True) + 7) // 8, dtype=torch.float64,
                       device=A0.device)

    def emulated():
        A.copy_(A0)
        X.copy_(B0)
        ca.calu_factor_mixed(A, b, tree, slices=7, exact=True, ipiv=ipiv, work=wemu, dev_info=info)
        ca.calu_getrs(A, ipiv, X, work=swork)

    ms, _ = timed(emulated, "fp64_emulated")
    out["fp64_emulated"] = {"ms": ms, "gflops": lu_flops / ms / 1e6, "berr": berr_of(X),
                            "speedup_vs_fp64": out["fp64"]["ms"] / ms,
                            "form": "calu_factor_mixed(7 exact digits) + calu_getrs: FP64-accurate update "
                                    "on the tensor cores"}
    # QR: least squares, plain FP64 vs the 7-digit tensor-core tree update
    qr_flops = 4.0 * n ** 3 / 3.0 + 3.0 * n * n * a.nrhs
    qb, qw = ca.ca_caqr_workspace(n, n, b, tree)
    qtree = torch.empty((qb + 7) // 8, dtype=torch.float64, device=A0.device)
    qwork = torch.empty((max(qw, ca.ca_geqrs_workspace(n, n, a.nrhs, b, tree)) + 7) // 8, dtype=torch.float64,
                        device=A0.device)
    _, qwm = ca.ca_caqr_mixed_workspace(n, n, b, tree, 7, True)
    qwmix = torch.empty((qwm + 7) // 8, dtype=torch.float64, device=A0.device)

    def qr_plain():
        A.copy_(A0)
        X.copy_(B0)
        ca.caqr_factor(A, b, tree, qtree=qtree, work=qwork, dev_info=info)
        ca.caqr_geqrs(A, b, tree, qtree, X, work=qwork)

    ms, _ = timed(qr_plain)
    out["qr_fp64"] = {"ms": ms, "gflops": qr_flops / ms / 1e6, "berr": berr_of(X),
                      "form": "caqr_factor + caqr_geqrs, FP64 DFMA tree update"}

    def qr_emulated():
        A.copy_(A0)
        X.copy_(B0)
        ca.caqr_factor_mixed(A, b, tree, slices=7, exact=True, qtree=qtree, work=qwmix, dev_info=info)
        ca.caqr_geqrs(A, b, tree, qtree, X, work=qwork)

    ms, _ = timed(qr_emulated, "qr_fp64_emulated")
    out["qr_fp64_emulated"] = {"ms": ms, "gflops": qr_flops / ms / 1e6, "berr": berr_of(X),
                               "speedup_vs_fp64": out["qr_fp64"]["ms"] / ms,
                               "form": "caqr_factor_mixed(7 exact digits) + caqr_geqrs: FP64-accurate tree "
                                       "update on the tensor cores"}
    del qwmix
    torch.cuda.empty_cache()
    qg, wg = ca.ca_gels_mixed_workspace(n, n, a.nrhs, b, tree, S, ex)
    qtg = torch.empty((qg + 7) // 8, dtype=torch.float64, device=A0.device)
    wgl = torch.empty((wg + 7) // 8, dtype=torch.float64, device=A0.device)

    def qr_mixed():
        return ca.caqr_gels_mixed(A0, B0, b, tree, slices=S, exact=ex, max_iter=10, tol=1e-14, QR=A, qtree=qtg,
                                  X=X, work=wgl, dev_info=info)

    ms, (_, it, be, _) = timed(qr_mixed, "qr_mixed_ir")
    out["qr_mixed_ir"] = {"ms": ms, "gflops": qr_flops / ms / 1e6, "iters": int(it.item()),
                          "ls_measure": float(be.item()), "berr": berr_of(X),
                          "x_rel_err": float(torch.linalg.norm(X - x_true) / torch.linalg.norm(x_true)),
                          "speedup_vs_fp64": out["qr_fp64"]["ms"] / ms,
                          "form": (f"caqr_gels_mixed: {S}-digit bf16 tensor-core tree update + refinement of "
                                   "the corrected semi-normal equations (double-double residual)")}
    del qtg, wgl
    for k, v in kernels_of.items():
        out[k]["kernels"] = v
    tc = kernels_of.get("mixed_factor", {}).get("gemm_tc")
    if tc and tc["ms"] > 0:
        # bf16 flops issued by the tensor-core update (2 M N K per digit
        # product, padded tile sizes) over its summed CUDA-event time
        ach = tc["gflop"] / tc["ms"]  # GFLOP per ms = TFLOP/s
        out["mixed_factor"]["roofline"] = {
            "kernel": "gemm_tc", "bound": "tensor", "achieved": ach, "unit": "TFLOP/s",
            "peak": BF16_TFLOPS, "frac": ach / BF16_TFLOPS,
            "peak_sustained": BF16_TFLOPS_SUSTAINED, "frac_of_sustained": ach / BF16_TFLOPS_SUSTAINED,
            "peak_source": f"cuBLAS bf16 GEMM, {BF16_SOURCE} (MEASURED_PEAKS.json: burst and sustained)",
            "work": "2 M N K x S (S + 1) / 2 bf16 flop per launch (exact digit products)"}
    return out


def other_configs(a, ca, torch, dev):
    """The other configurations of the workload family, each timed on its own
    (3 runs after a warm-up, CUDA events, the input restored between runs):
    the tall-skinny panels alone (TSLU and TSQR of 1,048,576 x 64 and
    8,388,608 x 32 N(0, 1) matrices, leaves of 256 rows, 4-level tree) with
    algorithmic HBM bytes (TSQR: A read, Y written = 16 m n; TSLU: A read
    twice, L written = 24 m n) and standard flops (TSQR 2 m n^2 - 2 n^3 / 3,
    TSLU m n^2 - n^3 / 3), and the small square case (CALU and CAQR of one
    1024 x 1024 matrix, b = 64, leaves of 128 rows, binary tree)."""
    out = {}
    gen = torch.Generator(device=dev).manual_seed(31)

    def timed(fn, A, A0, reps=3):
        A.copy_(A0)
        fn(A)
        torch.cuda.synchronize()
        best = []
        for _ in range(reps):
            A.copy_(A0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(A)
            e1.record()
            e1.synchronize()
            best.append(e0.elapsed_time(e1))
        return statistics.median(best)

    tree4 = ca.make_tree(256, [(4, 0), (8, 0), (0, 0)])
    for m, n in ((1048576, 64), (8388608, 32)):
        A0 = torch.randn(n, m, dtype=torch.float64, device=dev, generator=gen).t()
        A = torch.empty_like(A0)
        qb, wb = ca.ca_caqr_workspace(m, n, n, tree4)
        qt = torch.empty((qb + 7) // 8, dtype=torch.float64, device=dev)
        qw = torch.empty((wb + 7) // 8, dtype=torch.float64, device=dev)
        lw = torch.empty((ca.ca_calu_workspace(m, n, n, tree4) + 7) // 8, dtype=torch.float64, device=dev)
        ipiv = torch.empty(n, dtype=torch.int32, device=dev)
        info = torch.zeros(2, dtype=torch.int32, device=dev)
        ms_q = timed(lambda X: ca.tsqr(X, tree4, qtree=qt, work=qw, dev_info=info), A, A0)
        ms_l = timed(lambda X: ca.tslu(X, tree4, ipiv=ipiv, work=lw, dev_info=info), A, A0)
        fq, fl = 2.0 * m * n * n - 2.0 * n ** 3 / 3, m * n * n - n ** 3 / 3.0
        bq, bl = 16.0 * m * n, 24.0 * m * n
        out[f"panel_{m}x{n}"] = {
            "tsqr": {"ms": ms_q, "gflops": fq / ms_q / 1e6, "gbs": bq / ms_q / 1e6,
                     "frac_fp64": fq / ms_q / 1e6 / PEAKS["fp64"], "frac_hbm": bq / ms_q / 1e6 / HBM_GBS},
            "tslu": {"ms": ms_l, "gflops": fl / ms_l / 1e6, "gbs": bl / ms_l / 1e6,
                     "frac_fp64": fl / ms_l / 1e6 / PEAKS["fp64"], "frac_hbm": bl / ms_l / 1e6 / HBM_GBS}}
        del A0, A, qt, qw, lw
    n, b = 1024, 64
    t2 = ca.make_tree(128, [(0, 0)])
    A0 = torch.randn(n, n, dtype=torch.float64, device=dev, generator=gen).t()
    A = torch.empty_like(A0)
    ms_lu = timed(lambda X: ca.calu_factor(X, b, t2), A, A0)
    ms_qr = timed(lambda X: ca.caqr_factor(X, b, t2), A, A0)
    out["square_1024_b64"] = {"calu_ms": ms_lu, "calu_gflops": 2.0 * n ** 3 / 3 / ms_lu / 1e6,
                              "caqr_ms": ms_qr, "caqr_gflops": 4.0 * n ** 3 / 3 / ms_qr / 1e6}
    out["hbm_peak_gbs"] = HBM_GBS
    return out


OPERATOR_FORMS = [  # (name, panel width, leaf rows, levels, reduction operator)
    ("gepp", 32, 4096, [(0, 0)], []),
    ("calu", 64, 128, [(0, 0)], []),
    ("2d_ml_calu_depth1", 64, 128, [(0, 0)], [(16, 32)]),
    ("2d_ml_calu_depth2", 64, 256, [(0, 0)], [(32, 64), (8, 16)]),
]


def operator_diagnostics(a, ca, torch, dev, count=64, n=512):
    """Stability of the reduction operators on `count` seeded N(0, 1)
    matrices of order n, each form one batched launch: growth max|U| / max|A|,
    normwise backward error ||P A - L U||_F / ||A||_F, max |L| and the pivot
    threshold tau_min = 1 / max |L| (at step k the Schur complement's column
    is L(k:, k) U(k, k)), the componentwise backward error of a solve with
    the factors (median and worst over the sample), and the launch time.  GEPP
    is CALU with one leaf holding every row (blocked GEPP)."""
    gen = torch.Generator(device=dev).manual_seed(4242)
    A0 = [torch.randn(n, n, dtype=torch.float64, device=dev, generator=gen).t() for _ in range(count)]
    out = {"matrices": count, "n": n}
    for name, b, L, lv, op in OPERATOR_FORMS:
        mats = [A.clone() for A in A0]
        bf = ca.BatchedFactor(mats, ["lu"] * count, [b] * count, [ca.make_tree(L, lv, op)] * count)
        bf.run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for M, A in zip(mats, A0):
            M.copy_(A)
        e0.record()
        bf.run()
        e1.record()
        e1.synchronize()
        growth, berr, lmax, cberr = [], [], [], []
        xt = torch.ones(n, 1, dtype=torch.float64, device=dev)
        for i, (F, A) in enumerate(zip(mats, A0)):
            Lf = torch.tril(F, -1) + torch.eye(n, dtype=F.dtype, device=dev)
            U = torch.triu(F)
            perm = torch.arange(n, device=dev)
            for j, p in enumerate(bf.ipiv(i).cpu().tolist()):
                perm[[j, p - 1]] = perm[[p - 1, j]]
            growth.append(float(U.abs().max() / A.abs().max()))
            berr.append(float(torch.linalg.norm(A[perm] - Lf @ U) / torch.linalg.norm(A)))
            lmax.append(float(Lf.abs().max()))
            # componentwise backward error of a solve with these factors
            bb = A @ xt
            y = torch.linalg.solve_triangular(Lf, bb[perm], upper=False, unitriangular=True)
            x = torch.linalg.solve_triangular(U, y, upper=True)
            cberr.append(float(((bb - A @ x).abs() / (A.abs() @ x.abs() + bb.abs())).max()))
        out[name] = {"b": b, "leaf_rows": L, "operator": op, "ms": e0.elapsed_time(e1),
                     "growth_median": statistics.median(growth), "growth_max": max(growth),
                     "berr_median": statistics.median(berr), "berr_max": max(berr),
                     "lmax_max": max(lmax), "tau_min": 1.0 / max(lmax),
                     "componentwise_berr_max": max(cberr),
                     "nonzero_info": int((bf.info_all != 0).sum())}
    return out


OPERATOR_FORMS_8192 = [  # (name, panel width, leaf rows, levels, reduction operator)
    ("calu", 64, 256, [(0, 0)], []),
    ("2d_ml_calu_depth1", 64, 256, [(0, 0)], [(32, 64)]),
    ("2d_ml_calu_depth2", 64, 256, [(0, 0)], [(32, 64), (8, 16)]),
]


def operator_diagnostics_large(a, ca, torch, dev, n=8192):
    """The stability experiment of the multilevel CALU (Sec. 5.1) at the
    paper's order n = 8192 with its block sizes b = 64 / 32 / 8, in the
    single-matrix path (calu_factor): leaves of 256 rows under a binary tree
    (the paper's Pr3 = 16 leaves of 512 rows do not fit one CTA's shared
    memory), each node factored by CALU with b = 32 over 4 row blocks of 64
    (depth 1), whose nodes are factored by CALU with b = 8 over 4 blocks of 16
    (depth 2).  For each synthetic family (Gaussian N(0,1); A = U diag(s) V^T
    with cond 1e8, Haar U, V): growth max|U| / max|A|, ||P A - L U||_F /
    ||A||_F, tau_min = 1 / max|L| and the componentwise backward error of a
    solve, each also as a ratio to GEPP (torch.linalg.lu_factor, a library
    LU used here only as the reference of the ratios)."""
    from paper_1303_5837_gb300 import inputs
    out = {"n": n, "forms": {f[0]: {"b": f[1], "leaf_rows": f[2], "operator": f[4]} for f in OPERATOR_FORMS_8192}}
    g = torch.Generator(device=dev).manual_seed(58)
    fams = {"gaussian": torch.randn(n, n, dtype=torch.float64, device=dev, generator=g).t().contiguous().t()}
    U, V = haar_device(n, 59, dev), haar_device(n, 60, dev)
    s_ = torch.from_numpy(inputs.singular_values(n, 1e8)).to(dev)
    fams["cond1e8"] = ((U * s_) @ V.t()).t().contiguous().t()
    del U, V
    xt = torch.ones(n, 1, dtype=torch.float64, device=dev)

    def metrics(A, LU, perm):
        Lf = torch.tril(LU, -1) + torch.eye(n, dtype=LU.dtype, device=dev)
        Uf = torch.triu(LU)
        res = {"growth": float(Uf.abs().max() / A.abs().max()),
               "berr": float(torch.linalg.norm(A[perm] - Lf @ Uf) / torch.linalg.norm(A)),
               "tau_min": float(1.0 / Lf.abs().max())}
        bb = A @ xt
        y = torch.linalg.solve_triangular(Lf, bb[perm], upper=False, unitriangular=True)
        x = torch.linalg.solve_triangular(Uf, y, upper=True)
        res["componentwise_berr"] = float(((bb - A @ x).abs() / (A.abs() @ x.abs() + bb.abs())).max())
        return res

    def perm_of(ipiv):
        perm = np.arange(n)
        for i, p in enumerate(ipiv.cpu().numpy()):
            perm[i], perm[p - 1] = perm[p - 1], perm[i]
        return torch.from_numpy(perm).to(dev)

    for fname, A in fams.items():
        row = {}
        LUg, piv = torch.linalg.lu_factor(A)
        ref = metrics(A, LUg, perm_of(piv))
        row["gepp"] = ref
        del LUg
        for name, b, L, lv, op in OPERATOR_FORMS_8192:
            F = A.clone()
            t = ca.make_tree(L, lv, op)
            ca.calu_factor(F, b, t)  # warm-up of the shapes
            F.copy_(A)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ipiv, info = ca.calu_factor(F, b, t)
            e1.record()
            e1.synchronize()
            r = metrics(A, F, perm_of(ipiv))
            r["ms"] = e0.elapsed_time(e1)
            r["info"] = info.cpu().tolist()
            for k in ("growth", "berr", "componentwise_berr"):
                r[k + "_ratio_to_gepp"] = r[k] / ref[k] if ref[k] > 0 else None
            row[name] = r
            del F
        out[fname] = row
        torch.cuda.empty_cache()
    return out


BATCH_TABLES = {"f64": os.path.join(ROOT, "paper_1303_5837_gb300", "tuned_batch_f64.json"),
                "f32": os.path.join(ROOT, "paper_1303_5837_gb300", "tuned_batch_f32.json")}


def batched_run(a, ca, torch, dtype, dev, rank, world):
    """The batched workload: a.batch_count matrices (half square with n in
    [32, 512], half tall with m in [256, 8192] and n in {16, 32, 64, 128}),
    each factored by CALU and by CAQR, all in one persistent launch replayed
    from a CUDA graph; tile and tree shapes from the tuned table.  Inputs are
    seeded N(0, 1) drawn on the device (11 GB in FP64, larger than L2) and
    restored from a pristine copy before every (untimed) replay."""
    from paper_1303_5837_gb300 import tune
    tname = "f64" if dtype == torch.float64 else "f32"
    esz = 8 if dtype == torch.float64 else 4
    table = tune.load_table(BATCH_TABLES[tname])
    shapes, ops, bs, trees = tune.batch_items(2026 + rank, a.batch_count, table, esz)
    offs, tot = [], 0
    for m, n in shapes:
        offs.append(tot)
        tot += (m * n + 31) // 32 * 32          # 256-byte aligned starts
    flat = torch.empty(tot, dtype=dtype, device=dev)
    flat.normal_(generator=torch.Generator(device=dev).manual_seed(99 + rank))
    for i in range(1, len(shapes), 2):          # the CAQR item factors the CALU item's matrix
        m, n = shapes[i]
        flat[offs[i]: offs[i] + m * n].copy_(flat[offs[i - 1]: offs[i - 1] + m * n])
    pristine = flat.clone()
    views = [flat[o: o + m * n].view(n, m).t() for o, (m, n) in zip(offs, shapes)]
    bf = ca.BatchedFactor(views, ops, bs, [ca.make_tree(L, lv) for L, lv in trees])
    graph = bf.graph()
    flops = sum(tune.item_flops(op, m, n) for op, (m, n) in zip(ops, shapes))
    st = torch.cuda.current_stream()
    for _ in range(2):
        flat.copy_(pristine)
        graph.replay()
    torch.cuda.synchronize()
    bad = int((bf.info_all != 0).sum())
    barrier(world)
    times = []
    for _ in range(a.batch_steps):
        flat.copy_(pristine)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        graph.replay()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = allreduce_max(statistics.median(times), world)
    gflops = world * flops / (ms / 1e3) / 1e9
    out = {"matrices": a.batch_count, "items": len(shapes), "ms": ms, "gflops": gflops,
           "gflop_per_step": flops / 1e9, "launches_per_step": 1, "graph": True,
           "tuned": table is not None, "nonzero_info": bad, "bytes": tot * esz,
           "form": "ca_batched_factor: one CTA per matrix, LPT work queue, CALU + CAQR of every matrix"}
    pk = PEAKS["fp64"] if dtype == torch.float64 else PEAKS["fp32"]
    out["roofline"] = {"bound": "alu", "achieved": gflops / world, "peak": pk, "unit": "GFLOP/s",
                       "frac": gflops / world / pk, "peak_source": PEAKS["source"],
                       "note": ("FP64 DFMA pipe" if dtype == torch.float64 else
                                "FP32 FFMA pipe (the batched FP32 form uses no tensor cores)")}
    del views, bf, graph, flat, pristine
    torch.cuda.empty_cache()
    return out


SERVE_SIZES = [64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 6144, 8192]


def conditioned_rect_device(m, n, cond, seed, dev):
    """An m x n matrix (m = n or 4n) A = U diag(s) V^T with orthonormal
    columns in U, orthogonal V and s_i = cond^(-i/(n-1)) in a seeded order, on
    the device: U, V Haar (QR of Gaussians) up to n = 2048, above that
    Kronecker products of Haar factors (n = 64 n2)."""
    import torch
    from paper_1303_5837_gb300 import inputs
    g = torch.Generator(device=dev).manual_seed(seed)

    _load_torch_linalg()

    def q_of(r, c):
        Q, R = torch.linalg.qr(torch.randn(r, c, dtype=torch.float64, device=dev, generator=g))
        return Q * torch.sign(torch.diagonal(R))[None, :]

    if n <= 2048:
        U, V = q_of(m, n), q_of(n, n)
    else:
        n1, n2 = 64, n // 64
        U = torch.kron(q_of(m // n * n1, n1), q_of(n2, n2))
        V = torch.kron(q_of(n1, n1), q_of(n2, n2))
    s_ = torch.from_numpy(inputs.singular_values(n, cond)).to(dev)
    perm = torch.randperm(n, device=dev, generator=g)
    A = (U * s_[perm]) @ V.t()
    return A


def serving_run(a):
    """Open-loop Poisson streams of A x = b (CALU) and least-squares (CAQR,
    m = 4n) requests: n log-uniform in [64, a.serve_nmax] snapped to a pool
    of sizes, cond(A) log-uniform in [1, a.serve_cond_max], 1-16 right-hand
    sides; the same a.serve_count requests at each rate of a.serve_rates,
    replayed in real time into (1) the plain per-request loop (one stream,
    arrival order, no overlap), (2) the continuous-batching server in FP64
    and (3) the server with the mixed forms.  Matrices come from a
    pre-generated pool, one per (kind, size), generated untimed."""
    import torch
    from paper_1303_5837_gb300 import serve
    dev = torch.device("cuda", torch.cuda.current_device())
    rates = [float(x) for x in a.serve_rates.split(",") if x]
    sizes = [s_ for s_ in SERVE_SIZES if s_ <= a.serve_nmax]
    works = {r: serve.poisson_workload(r, 0.0, seed=11, nmax=a.serve_nmax, count=a.serve_count, sizes=sizes)
             for r in rates}
    pool = {}
    t_pool = time.perf_counter()
    for work in works.values():
        for _, kind, m, n, nrhs in work:
            key = (kind, n)
            if key in pool:
                continue
            g = np.random.default_rng(1000 * n + (7 if kind == "ls" else 0))
            cond = float(10.0 ** g.uniform(0.0, np.log10(a.serve_cond_max)))
            A = conditioned_rect_device(m, n, cond, 17 * n + (3 if kind == "ls" else 0), dev)
            pool[key] = (np.asfortranarray(A.cpu().numpy()), g.standard_normal((m, 16)), cond)
            del A
    torch.cuda.empty_cache()
    out = {"rates_per_s": rates, "requests_per_rate": a.serve_count, "n_sizes": sizes,
           "m": "n (LU) or 4n (least squares)", "cond_range": [1.0, a.serve_cond_max],
           "pool_matrices": len(pool), "pool_seconds": time.perf_counter() - t_pool, "slots": a.serve_slots,
           "forms": {"plain": "one stream, one request at a time in arrival order, FP64 "
                              "(calu_factor + calu_getrs / caqr_factor + caqr_geqrs)",
                     "fp64": "continuous-batching server, FP64 factorizations",
                     "mixed": "continuous-batching server, LU by calu_gesv_mixed (4 digits, refine auto), "
                              "least squares by caqr_gels_mixed (4 digits, refinement)"},
           "sweep": {}}
    for rate, work in works.items():
        row = {}
        items = [(t, kind, pool[(kind, n)][0], pool[(kind, n)][1][:, :nrhs]) for t, kind, m, n, nrhs in work]
        done = serve.run_plain(items, form="fp64", device=dev.index)
        st = serve.latency_stats([r for r in done if r.status == "done"])
        st["failed"] = sum(1 for r in done if r.status != "done")
        row["plain"] = st
        for form in ("fp64", "mixed"):
            srv = serve.SolveServer(hbm_budget=64 << 30, slots=a.serve_slots, form=form, device=dev.index)
            try:
                t0 = time.perf_counter()
                reqs = []
                for t, kind, A, Bm in items:
                    now = time.perf_counter() - t0
                    if t > now:
                        time.sleep(t - now)
                    reqs.append(srv.submit(kind, A, Bm))
                srv.drain(timeout=900)
                st = srv.stats()
                st["failed"] = sum(1 for r in reqs if r.status == "failed")
            finally:
                srv.close()
            row[form] = st
        row["speedup_solves_per_s"] = {f: row[f]["solves_per_s"] / row["plain"]["solves_per_s"]
                                      for f in ("fp64", "mixed") if row["plain"].get("solves_per_s")}
        out["sweep"][str(int(rate))] = row
    return out


def conditioned_device(n, cond, seed, dev):
    """A = U diag(s) V^T in FP64 on the device, s log-spaced from 1 to 1/cond
    in a seeded order; U and V Haar orthogonal (QR of a seeded Gaussian on
    the device, signs of R folded in; input generation, untimed)."""
    import torch
    from paper_1303_5837_gb300 import inputs
    if n < 4096:
        return torch.from_numpy(np.ascontiguousarray(inputs.conditioned(n, cond, seed).T)).to(dev).t()
    U = haar_device(n, 7 * seed + 1, dev)
    V = haar_device(n, 7 * seed + 2, dev)
    s = torch.from_numpy(inputs.singular_values(n, cond)).to(dev)
    perm = torch.from_numpy(np.random.Generator(np.random.PCG64(seed)).permutation(n)).to(dev)
    A = (U * s[perm]) @ V.t()
    del U, V
    return A.t().contiguous().t()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    """Max over ranks (the timing rule); on the CUDA device for NCCL, on the
    host for gloo."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.derive_traffic:
        print_traffic_line(a)
        return
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    run_ours(a, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
