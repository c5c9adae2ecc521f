"""The serving loop's scheduling on the host (no GPU): requests are admitted in
arrival order only while their HBM footprint fits the budget and a slot is
free, oversized requests are rejected, work overlaps across slots, and the
latency statistics cover every completed request."""
import threading
import time

import numpy as np

from paper_1303_5837_gb300 import serve


def test_admission_by_footprint_and_slots():
    active = []
    peak = {"n": 0, "bytes": 0}
    lock = threading.Lock()

    def fake_execute(r, ctx):
        with lock:
            active.append(r)
            peak["n"] = max(peak["n"], len(active))
            peak["bytes"] = max(peak["bytes"], sum(x.footprint for x in active))
        time.sleep(0.02)
        with lock:
            active.remove(r)
        return np.zeros((r.A.shape[1], r.B.shape[1]))

    n = 256
    one = serve.footprint("lu", n, n, 1, 128, serve.B.make_tree(256, [(4, 0), (0, 0)]))
    srv = serve.SolveServer(hbm_budget=int(2.5 * one), slots=4, execute=fake_execute)
    try:
        reqs = [srv.submit("lu", np.eye(n), np.ones(n)) for _ in range(8)]
        huge = srv.submit("lu", np.eye(2 * n), np.ones(2 * n))  # 4x the footprint: over budget
        srv.drain(timeout=30)
    finally:
        srv.close()
    assert all(r.status == "done" for r in reqs)
    assert huge.status == "rejected"
    assert peak["n"] == 2                     # the budget holds two at a time, not four slots' worth
    assert peak["bytes"] <= srv.budget
    assert srv.max_used <= srv.budget
    st = srv.stats()
    assert st["completed"] == 8 and st["rejected"] == 1
    assert st["p99_s"] >= st["p50_s"] > 0


def test_poisson_workload_shapes():
    w = serve.poisson_workload(rate=200.0, duration=2.0, seed=1, nmin=64, nmax=2048)
    assert 300 < len(w) < 500
    ts = [x[0] for x in w]
    assert ts == sorted(ts) and ts[-1] <= 2.0
    for t, kind, m, n, nrhs in w:
        assert 64 <= n <= 2048 and 1 <= nrhs <= 16
        assert m == (4 * n if kind == "ls" else n)


def test_failed_request_does_not_stop_the_server():
    def flaky(r, ctx):
        if r.B[0, 0] < 0:
            raise RuntimeError("planted failure")
        return np.zeros((1, 1))

    srv = serve.SolveServer(hbm_budget=1 << 40, slots=2, execute=flaky)
    try:
        bad = srv.submit("lu", np.eye(64), -np.ones(64))
        good = srv.submit("lu", np.eye(64), np.ones(64))
        srv.drain(timeout=30)
    finally:
        srv.close()
    assert bad.status == "failed" and "planted" in bad.error
    assert good.status == "done"


def test_cancel_a_pending_request():
    """A request still waiting for a slot can be cancelled: it finishes as
    "cancelled" and never reaches the executor; a running one cannot be
    cancelled and completes; later requests are served in order."""
    seen = []
    started = threading.Event()

    def slow(r, ctx):
        seen.append(r)
        started.set()
        time.sleep(0.3)
        return np.zeros((1, 1))

    srv = serve.SolveServer(hbm_budget=1 << 40, slots=1, execute=slow)
    try:
        first = srv.submit("lu", np.eye(64), np.ones(64))
        assert started.wait(10)
        second = srv.submit("lu", np.eye(64), np.ones(64))
        third = srv.submit("lu", np.eye(64), np.ones(64))
        assert not srv.cancel(first)           # running: not interrupted
        assert srv.cancel(second)              # still waiting for the slot
        assert not srv.cancel(second)          # only once
        assert second.done.is_set() and second.status == "cancelled"
        srv.drain(timeout=30)
        assert not srv.cancel(third)           # finished
    finally:
        srv.close()
    assert first.status == "done" and third.status == "done"
    assert second not in seen and seen == [first, third]
    st = srv.stats()
    assert st["completed"] == 2 and st["cancelled"] == 1 and st["rejected"] == 0


def test_library_status_fails_the_request():
    """A zero pivot, a status bit of dev_info (NaN/Inf, tensor-core or solve
    timeout), a triangular solve that gave up, or a non-finite backward
    error turns the request into a failure with the reason; the server
    keeps serving."""
    import pytest
    with pytest.raises(RuntimeError, match="singular"):
        serve.check_result([5, 0], False)
    with pytest.raises(RuntimeError, match="0x10"):
        serve.check_result([0, 16], False)
    with pytest.raises(RuntimeError, match="gave up"):
        serve.check_result([0, 0], True)
    with pytest.raises(RuntimeError, match="backward error"):
        serve.check_result([0, 0], False, float("nan"))
    serve.check_result([0, 0], False, 1e-15)

    def execute(r, ctx):
        serve.check_result([0, int(r.B[0, 0])], bool(r.B[1, 0]))
        return np.zeros((r.A.shape[1], 1))

    srv = serve.SolveServer(hbm_budget=1 << 40, slots=2, execute=execute)
    try:
        timeout_bit = srv.submit("lu", np.eye(8), np.r_[16.0, 0.0, np.zeros(6)])
        gave_up = srv.submit("lu", np.eye(8), np.r_[0.0, 1.0, np.zeros(6)])
        ok = srv.submit("lu", np.eye(8), np.zeros(8))
        srv.drain(timeout=30)
    finally:
        srv.close()
    assert timeout_bit.status == "failed" and "0x10" in timeout_bit.error
    assert gave_up.status == "failed" and "gave up" in gave_up.error
    assert ok.status == "done" and srv.stats()["completed"] == 1


def test_max_on_device_counts_overlapping_intervals():
    srv = serve.SolveServer(hbm_budget=1 << 40, slots=1, execute=lambda r, c: np.zeros((1, 1)))
    try:
        for iv in [(0.0, 5.0), (1.0, 2.0), (1.5, 6.0), (7.0, 8.0)]:
            r = serve.Request("lu", np.eye(2), np.ones((2, 1)))
            r.gpu_ms = iv
            srv.completed.append(r)
        assert srv.max_on_device() == 3
    finally:
        srv.close()
