"""Host-side logic of the batched path (no GPU): the workload's shape
distribution, size classes, the tuner's candidate filter and table files,
and the ctypes layout of the C-ABI structs against the C compiler's."""
import ctypes
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1303_5837_gb300 import tune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batch_shapes_follow_the_workload():
    shapes = tune.batch_shapes(2026, 4096)
    sq = [s for i, s in enumerate(shapes) if i % 2 == 0]
    tall = [s for i, s in enumerate(shapes) if i % 2 == 1]
    assert len(sq) == len(tall) == 2048
    assert all(m == n and 32 <= n <= 512 for m, n in sq)
    assert all(256 <= m <= 8192 and n in (16, 32, 64, 128) for m, n in tall)
    # roughly uniform: every quarter of the ranges is populated
    ns = np.array([n for _, n in sq])
    assert all(((ns >= lo) & (ns < lo + 120)).sum() > 300 for lo in (32, 152, 272, 392))
    assert len({n for _, n in tall}) == 4
    # seeded: the same seed gives the same batch
    assert tune.batch_shapes(2026, 64) == tune.batch_shapes(2026, 64)


def test_batch_items_pair_every_matrix_with_lu_and_qr():
    shapes, ops, bs, trees = tune.batch_items(7, 50)
    assert len(shapes) == 100 and ops == ["lu", "qr"] * 50
    assert shapes[0::2] == shapes[1::2]
    for (m, n), b, (L, lv) in zip(shapes, bs, trees):
        assert 1 <= b <= 128 and L >= min(b, m, n)
        assert lv in tune.TREES.values()


def test_item_flops_are_the_standard_counts():
    assert tune.item_flops("lu", 300, 300) == pytest.approx(2 * 300 ** 3 / 3)
    assert tune.item_flops("lu", 1000, 64) == pytest.approx(1000 * 64 ** 2 - 64 ** 3 / 3)
    assert tune.item_flops("qr", 1000, 64) == pytest.approx(2 * 1000 * 64 ** 2 - 2 * 64 ** 3 / 3)


def test_classes_and_candidates():
    assert tune.class_of("lu", 300, 300) == ("lu", 512, 1)
    assert tune.class_of("qr", 8000, 64) == ("qr", 64, 64)
    for op, m, n in [("lu", 512, 512), ("qr", 8192, 128), ("lu", 256, 16), ("qr", 40, 40)]:
        cands = tune.candidates(op, m, n)
        assert cands, (op, m, n)
        for b, L, name in cands:
            assert L >= min(b, m, n)
            # a node tile (leaf rows or a merge) fits the shared-memory budget
            assert tune._node_fits(m, n, b, L, tune.TREES[name], 8)
        assert tune._node_fits(m, n, *tune.default_config(op, m, n)[:2], tune.TREES["binary"], 8)
    # a 128-wide FP64 binary merge (257 x 128 doubles) does not fit; FP32 does
    assert not tune._node_fits(4096, 128, 128, 128, tune.TREES["binary"], 8)
    assert tune._node_fits(4096, 128, 128, 128, tune.TREES["binary"], 4)


def test_table_round_trip(tmp_path):
    table = {("lu", 512, 1): (32, 512, "flat"), ("qr", 64, 64): (16, 256, "flat4")}
    path = tmp_path / "t.json"
    tune.save_table(str(path), table, {"dtype": "f64"})
    assert tune.load_table(str(path)) == table
    assert json.load(open(path))["meta"]["dtype"] == "f64"
    assert tune.load_table(str(tmp_path / "missing.json")) is None
    # the committed tables parse and name known trees
    for dt in ("f64", "f32"):
        t = tune.load_table(os.path.join(ROOT, "paper_1303_5837_gb300", f"tuned_batch_{dt}.json"))
        assert t and all(v[2] in tune.TREES for v in t.values())


C_LAYOUT = r"""
#include <stdio.h>
#include <stddef.h>
#include "ca_gb300.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(ca_tree_t), offsetof(ca_tree_t, op_depth), offsetof(ca_tree_t, op_b),
         offsetof(ca_tree_t, op_leaf_rows));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(ca_batch_item_t), offsetof(ca_batch_item_t, A),
         offsetof(ca_batch_item_t, qtree), offsetof(ca_batch_item_t, info), offsetof(ca_batch_item_t, b),
         offsetof(ca_batch_item_t, tree));
  return 0;
}
"""


def test_ctypes_structs_match_the_c_header(tmp_path):
    gcc = shutil.which("gcc")
    cuda_inc = "/usr/local/cuda/include"
    if not gcc or not os.path.isdir(cuda_inc):
        pytest.skip("gcc or the CUDA headers are missing")
    src = tmp_path / "layout.c"
    src.write_text(C_LAYOUT)
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    from paper_1303_5837_gb300 import _binding as B
    T, I = B.ca_tree_t, B.ca_batch_item_t
    assert [int(x) for x in out[0].split()] == [ctypes.sizeof(T), T.op_depth.offset, T.op_b.offset,
                                                T.op_leaf_rows.offset]
    assert [int(x) for x in out[1].split()] == [ctypes.sizeof(I), I.A.offset, I.qtree.offset, I.info.offset,
                                                I.b.offset, I.tree.offset]
