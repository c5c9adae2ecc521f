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


def batch_workload(seed: int, count: int, table=None, esz: int = 8):
    """The batch: `count` matrices from ``batch_shapes``, each factored by
    CALU and by CAQR (2 * count items).  Returns (host matrices, ops, panel
    widths, trees as (leaf_rows, levels)); shapes from ``table`` (class ->
    (b, leaf_rows, tree name)) or the untuned defaults."""
    shapes = batch_shapes(seed, count)
    base = batch_matrices(shapes, seed)
    mats, ops, bs, trees = [], [], [], []
    for A in base:
        m, n = A.shape
        for op in ("lu", "qr"):
            cfg = (table or {}).get(class_of(op, m, n)) or default_config(op, m, n, esz)
            b, L, name = cfg
            mats.append(A.copy(order="F"))
            ops.append(op)
            bs.append(int(b))
            trees.append((int(L), TREES[name]))
    return mats, ops, bs, trees


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
        for L in (64, 128, 256):
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
            mats = [torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda", self.dtype).t()
                    for A in batch_matrices(samp, seed + 7)]
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
