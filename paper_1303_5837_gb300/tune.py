"""Batched workloads and the autotuner of their tile and tree shapes.

``batch_shapes`` draws the uneven batch of many small factorizations (square
matrices with n uniform in [32, 512], tall-skinny ones with m uniform in
[256, 8192] and n in {16, 32, 64, 128}); ``batch_matrices`` fills them with
seeded iid N(0, 1) entries.

The tuner groups the items of a batch into classes (operation, n rounded up
to a power of two, rows per column rounded to a power of two), and for each
class times every candidate shape -- panel width b, leaf rows and tree
(binary over all leaves, one flat merge of all leaves, flat groups of 4 then
binary) -- on a sample of the class's matrices with one batched launch per
candidate (CUDA events around the launch, the sample restored from a pristine
copy between trials), and keeps the fastest.  Only host-side orchestration
lives here: every trial is a call of the C-ABI (``ca_batched_factor``).
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs

BIN, FLAT = 0, 1
TREES = {
    "binary": [(0, BIN)],
    "flat": [(0, FLAT)],
    "flat4": [(4, FLAT), (0, BIN)],
}
SMEM_REGION = {8: 200 * 1024, 4: 200 * 1024}   # bytes of a node tile the kernel can hold (about)


def batch_shapes(seed: int, count: int):
    """(m, n) of `count` matrices: half square (n ~ U[32, 512]), half tall
    (m ~ U[256, 8192], n in {16, 32, 64, 128})."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        if i % 2 == 0:
            n = int(g.integers(32, 513))
            out.append((n, n))
        else:
            m = int(g.integers(256, 8193))
            n = int(g.choice([16, 32, 64, 128]))
            out.append((m, n))
    return out


def batch_matrices(shapes, seed: int):
    return [inputs.gaussian(m, n, seed * 100003 + i) for i, (m, n) in enumerate(shapes)]


def batch_items(seed: int, count: int, table=None, esz: int = 8):
    """Items of the batch: `count` matrices from ``batch_shapes``, each
    factored by CALU and by CAQR (2 * count items).  Returns (shapes, ops,
    panel widths, trees as (leaf_rows, levels)); shapes from ``table``
    (class -> (b, leaf_rows, tree name)) or the untuned defaults."""
    shapes, ops, bs, trees = [], [], [], []
    for m, n in batch_shapes(seed, count):
        for op in ("lu", "qr"):
            cfg = (table or {}).get(class_of(op, m, n)) or default_config(op, m, n, esz)
            b, L, name = cfg
            shapes.append((m, n))
            ops.append(op)
            bs.append(int(b))
            trees.append((int(L), TREES[name]))
    return shapes, ops, bs, trees


def batch_workload(seed: int, count: int, table=None, esz: int = 8):
    """``batch_items`` with host matrices (seeded iid N(0, 1); the CALU and
    the CAQR item of a matrix get the same values)."""
    shapes, ops, bs, trees = batch_items(seed, count, table, esz)
    base = batch_matrices(shapes[::2], seed)
    mats = [base[i // 2].copy(order="F") for i in range(len(shapes))]
    return mats, ops, bs, trees


def item_flops(op: str, m: int, n: int) -> float:
    """Standard flop counts: LU m n^2 - n^3 / 3 (m >= n), QR 2 m n^2 - 2 n^3 / 3."""
    if op == "lu":
        k = min(m, n)
        return 2.0 * (m * n * k - (m + n) * k * k / 2.0 + k ** 3 / 3.0)
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def load_table(path: str):
    """Tuned table from JSON ({"op,n,ratio": [b, leaf_rows, tree]})."""
    import json
    import os
    if not os.path.exists(path):
        return None
    raw = json.load(open(path))
    out = {}
    for k, v in raw.get("table", {}).items():
        op, nb, ratio = k.split(",")
        out[(op, int(nb), int(ratio))] = (int(v[0]), int(v[1]), str(v[2]))
    return out


def save_table(path: str, table: dict, meta: dict):
    import json
    raw = {"meta": meta, "table": {f"{k[0]},{k[1]},{k[2]}": list(v) for k, v in sorted(table.items())}}
    with open(path, "w") as f:
        json.dump(raw, f, indent=1, sort_keys=True)


def _node_fits(m: int, n: int, b: int, L: int, levels, esz: int) -> bool:
    bk = min(b, m, n)
    if L < bk or L < 1:
        return False
    if n > bk and bk > 64:
        return False
    nl = -(-m // L)
    rows = min(L, m)
    # largest merge: fan-in x bk rows
    for f, style in levels[:-1]:
        if style == FLAT:
            rows = max(rows, min(f, nl) * bk)
        else:
            rows = max(rows, 2 * bk)
        nl = -(-nl // max(f, 1))
    last_style = levels[-1][1]
    rows = max(rows, (nl * bk) if last_style == FLAT else (2 * bk if nl > 1 else rows))
    return rows <= 1024 and (rows | 1) * bk * esz <= SMEM_REGION[esz]


def candidates(op: str, m: int, n: int, esz: int = 8):
    """Candidate (b, leaf_rows, tree name) shapes of one matrix."""
    out = []
    k = min(m, n)
    bs = sorted({b for b in (16, 32, 64) if b <= max(16, k)} | ({k} if k <= 128 else set()))
    for b in bs:
        for L in (64, 128, 256, 512):
            if L < min(b, k):
                continue
            for name, lv in TREES.items():
                if _node_fits(m, n, b, L, lv, esz):
                    out.append((b, L, name))
    return out


def default_config(op: str, m: int, n: int, esz: int = 8):
    """Untuned shape: panel width 32 (square) or the matrix width (tall, up to
    what one CTA holds), 128- or 256-row leaves, binary tree."""
    if m == n:
        b = 32 if n <= 256 else 64
        return b, 128, "binary"
    for b in (n, 64, 32):
        for L in (256, 128):
            if _node_fits(m, n, b, L, TREES["binary"], esz):
                return b, L, "binary"
    return 16, 64, "binary"


def class_of(op: str, m: int, n: int):
    nb = 1 << max(0, math.ceil(math.log2(max(n, 1))))
    ratio = 1 << max(0, round(math.log2(max(m / max(n, 1), 1))))
    return (op, nb, min(ratio, 64))


class Tuner:
    """Picks the fastest (b, leaf_rows, tree) per class by timing batched
    launches on the GPU.  ``table`` maps a class to its choice."""

    def __init__(self, torch_mod, dtype, sample: int = 304, reps: int = 1):
        self.torch = torch_mod
        self.dtype = dtype
        self.esz = 8 if dtype == torch_mod.float64 else 4
        self.sample = sample
        self.reps = reps
        self.table: dict = {}
        self.trials: dict = {}

    def config(self, op: str, m: int, n: int):
        return self.table.get(class_of(op, m, n)) or default_config(op, m, n, self.esz)

    def tune(self, ops, shapes, seed: int = 1):
        from . import _binding as B
        torch = self.torch
        classes: dict = {}
        for op, (m, n) in zip(ops, shapes):
            classes.setdefault(class_of(op, m, n), []).append((m, n))
        g = np.random.default_rng(seed)
        for cls, members in sorted(classes.items()):
            op = cls[0]
            idx = g.choice(len(members), min(self.sample, len(members)), replace=False)
            samp = [members[i] for i in idx]
            gen = torch.Generator(device="cuda").manual_seed(seed + 7)
            mats = [torch.randn(n, m, dtype=self.dtype, device="cuda", generator=gen).t() for m, n in samp]
            pristine = [A.clone() for A in mats]
            # candidates valid for every sampled shape
            common = None
            for m, n in samp:
                c = set(candidates(op, m, n, self.esz))
                common = c if common is None else common & c
            best, results = None, {}
            for b, L, name in sorted(common or []):
                try:
                    bf = B.BatchedFactor(mats, [op] * len(mats), [b] * len(mats),
                                         [B.make_tree(L, TREES[name])] * len(mats))
                except B.CaError:
                    continue
                times = []
                for _ in range(self.reps + 1):
                    for A, P in zip(mats, pristine):
                        A.copy_(P)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    bf.run()
                    e1.record()
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                t = min(times[1:])
                results[(b, L, name)] = t
                if best is None or t < results[best]:
                    best = (b, L, name)
            if best is not None:
                self.table[cls] = best
                self.trials[cls] = results
        return self.table


def main(argv=None):
    """Tune the batch of ``batch_items`` on the current GPU and write the
    table (python -m paper_1303_5837_gb300.tune --dtype f64 --out FILE)."""
    import argparse
    import time

    import torch
    p = argparse.ArgumentParser()
    p.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    p.add_argument("--count", type=int, default=4096)
    p.add_argument("--seed", type=int, default=2026)
    p.add_argument("--sample", type=int, default=304)
    p.add_argument("--out", required=True)
    a = p.parse_args(argv)
    dt = torch.float64 if a.dtype == "f64" else torch.float32
    shapes, ops, _, _ = batch_items(a.seed, a.count)
    t0 = time.time()
    tu = Tuner(torch, dt, sample=a.sample)
    table = tu.tune(ops, shapes, seed=a.seed)
    meta = {"dtype": a.dtype, "count": a.count, "seed": a.seed, "sample": a.sample,
            "seconds": time.time() - t0, "device": torch.cuda.get_device_name(),
            "trials": {f"{k[0]},{k[1]},{k[2]}": {f"{b},{L},{t}": ms for (b, L, t), ms in v.items()}
                       for k, v in tu.trials.items()}}
    save_table(a.out, table, meta)
    print(f"tuned {len(table)} classes in {meta['seconds']:.1f} s -> {a.out}")


if __name__ == "__main__":
    main()
