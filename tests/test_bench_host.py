"""Host logic of bench.py that needs no GPU: the reduction-tree option and the
lookup of committed DRAM counters (profiles/traffic.txt), which must only be
used for the kernel code and the plan of launches they were taken on."""
import hashlib

import pytest

import bench


def test_parse_tree():
    assert bench.parse_tree("4f,0f") == [(4, 1), (0, 1)]
    assert bench.parse_tree("4b,0b") == [(4, 0), (0, 0)]
    assert bench.parse_tree(bench.BENCH_TREE)[-1][0] == 0
    for bad in ("4x,0b", "4b", "b,0b", ""):
        with pytest.raises(ValueError):
            bench.parse_tree(bad)
    assert "flat" in bench.describe_tree([(4, 1), (0, 1)])


def test_source_region(tmp_path):
    f = tmp_path / "k.cu"
    f.write_text("a\n// @region K\nbody 1\nbody 2\n// @endregion K\ntail\n")
    assert bench.source_text(str(tmp_path), "k.cu#K") == b"body 1\nbody 2\n"
    assert bench.source_text(str(tmp_path), "k.cu") == f.read_bytes()
    assert bench.source_text(str(tmp_path), "k.cu#missing") == b""


def test_traffic_key_matches_current_kernel_and_plan():
    plan = f"16384/128/{bench.BENCH_LEAF_ROWS}/{bench.BENCH_TREE}/320"
    v = bench.traffic_for("tree_apply", plan)
    assert v is not None and v > 0
    # another plan of launches (or another kernel) gets no figure
    assert bench.traffic_for("tree_apply", "16384/128/1024/4b,0b/496") is None
    assert bench.traffic_for("gemm_fp64", plan) is None


def test_traffic_key_detects_a_changed_kernel(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1303_5837_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("// @region K\nint x;\n// @endregion K\n")
    h = hashlib.sha256(b"int x;\n").hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.txt").write_text(f"kern k.cu#K {h} 1e6 plan=P note\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("kern", "P") == 1e6
    (csrc / "k.cu").write_text("// @region K\nint y;\n// @endregion K\n")
    assert bench.traffic_for("kern", "P") is None


def test_clock_rejection_rule():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 100}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(dict(ok, reasons=["sw_power_cap"]))            # kept, noted
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1500.0, reasons=["sw_power_cap"]))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))                            # stuck low, no reason
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                      "reasons": ["nvidia-smi unavailable"]})


@pytest.mark.parametrize("levels", ["0b", "0f", "4b,0b", "4f,0f", "2b,4b,0b", "3f,0b", "8f,0f", "2f,3b,0f"])
def test_tree_rounds_match_the_oracle_counts(levels):
    """The benchmark's replica of the library's merge rounds merges as many
    nodes as the oracle's (independent) tree plan, for ragged leaf counts."""
    import oracle
    lv = bench.parse_tree(levels)
    for nl in list(range(1, 40)) + [64, 97, 128, 513]:
        merges = sum(1 for rnd in bench.tree_rounds(nl, lv) for c in rnd if c >= 2)
        _, nm = oracle.tree_counts(nl * 64, oracle.make_tree(64, lv))
        assert merges == nm, (levels, nl)
        # every round's inputs are the previous round's outputs
        n_in = nl
        for rnd in bench.tree_rounds(nl, lv):
            assert sum(rnd) == n_in
            n_in = len(rnd)
        assert n_in == 1


def test_tree_update_plan_matches_the_measured_launch_counts():
    """Launch counts per step of the benchmark (n = 16384, b = 128, 1024-row
    leaves, one right-hand side) as the library's own counters reported them
    on the GPU: 320 wide / 709 narrow with flat merges of 4, 496 / 1061 with
    binary merges in groups of 4."""
    for tree, wide, narrow in (("4f,0f", 320, 709), ("4b,0b", 496, 1061)):
        d = bench.derive_traffic(14.54, 8.22, 16384, 128, 1024, bench.parse_tree(tree))
        assert (d["wide_launches"], d["narrow_launches"]) == (wide, narrow)
    d = bench.derive_traffic(1.0, 0.0, 6144, 128, 1024, bench.parse_tree("4f,0f"))
    ls = bench.tree_update_launches(6144, 128, 1024, bench.parse_tree("4f,0f"), 1)
    # panel 0 at n = 6144: the look-ahead update (narrow: 6 leaves x 4 tiles < 152
    # SMs), then the wide leaf launch of the other 5888 columns and two merge rounds
    assert [k for k, _, _ in ls[:6]] == ["tree_narrow"] * 3 + ["tree_apply"] * 3
    assert ls[3] == ("tree_apply", True, 6144 * 5888)
    assert ls[4] == ("tree_apply", False, 6 * 128 * 5888) and ls[5] == ("tree_apply", False, 2 * 128 * 5888)


def test_committed_traffic_line_is_the_derived_one():
    import subprocess
    import sys
    out = subprocess.run([sys.executable, "bench.py", "--derive-traffic", "14.54,8.22"],
                         cwd=bench.ROOT, capture_output=True, text=True, check=True).stdout
    committed = open(f"{bench.ROOT}/profiles/traffic.txt").read()
    assert out == committed


def test_reference_arm_line_follows_the_contract():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the contract's keys, on the main arm's metric and config."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--ref-n", "128"], cwd=bench.ROOT, capture_output=True, text=True, check=True,
                         timeout=300).stdout.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GFLOP/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0 and d["higher_is_better"] is True
    assert "workload" in d["config"] and d["config"]["sample_n"] == 128
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    import os
    import subprocess
    import sys
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-n", "64"], cwd=bench.ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_all_cores_oracle_baseline():
    """The oracle on every host core at once: spawned processes (safe after
    CUDA use), started together, aggregate throughput over the common span."""
    import argparse
    a = argparse.Namespace(cond=1e6, nrhs=1, b=64, leaf=128, tree="0b", cpu_n=128)
    d = bench.cpu_baseline_all_cores(a, cores=2)
    assert d is not None and d["cores"] == 2 and d["kind"] == "oracle"
    assert d["value"] > 0 and d["seconds"] > 0 and "2 concurrent copies" in d["sample"]
