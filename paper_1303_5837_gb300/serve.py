"""Continuous-batching solve server on one GPU.

Requests (A x = b by CALU + getrs, or least squares by CAQR + geqrs) arrive
at any time.  A scheduler thread admits them in arrival order as soon as a
slot is free and their HBM footprint (matrix, right-hand sides, solution and
the library's workspace, sized by the C-ABI workspace queries) fits in the
remaining budget; a request larger than the whole budget is rejected.  Each
slot is a worker thread with its own CUDA stream, so admitted requests run
concurrently on the device while later ones wait.  Factors stay on the device
for the life of a request; the result comes back to the host.  A request can
be cancelled until it is admitted; one that runs is never interrupted.

Every computation goes through the C-ABI (``_binding``); this module only
schedules, allocates (torch caching allocator) and moves data.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import _binding as B

LU, LS = "lu", "ls"


@dataclass(eq=False)  # requests compare by identity
class Request:
    kind: str                   # "lu" (square A x = b) or "ls" (least squares, m >= n)
    A: np.ndarray               # host, column-major float64
    B: np.ndarray               # host, m x nrhs
    arrival: float = 0.0
    footprint: int = 0
    status: str = "pending"     # pending, running, done, rejected, failed, cancelled
    X: np.ndarray | None = None
    t_done: float = 0.0
    error: str = ""
    berr: float = 0.0           # mixed LU: backward error reached by refinement
    gpu_ms: tuple = ()          # (start, end) on the device, ms after the server's reference event
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def footprint(kind: str, m: int, n: int, nrhs: int, b: int, tree, form: str = "fp64") -> int:
    """Device bytes a request holds while it runs."""
    mats = 8 * (m * n + 2 * m * nrhs)
    if kind == LU:
        if form == "mixed":
            w = B.ca_gesv_mixed_workspace(n, nrhs, b, tree, 4, True, "auto")
            return mats + 8 * n * n + w + 4 * n + 4096
        w = B.ca_calu_workspace(m, n, b, tree) + B.ca_getrs_workspace(n, nrhs)
        return mats + w + 4 * n + 4096
    if form == "mixed":
        q, w = B.ca_gels_mixed_workspace(m, n, nrhs, b, tree, 4, True)
        return mats + 8 * m * n + q + w + 4096
    q, w = B.ca_caqr_workspace(m, n, b, tree)
    w = max(w, B.ca_geqrs_workspace(m, n, nrhs, b, tree))
    return mats + q + w + 4096


class SolveServer:
    """``form``: "fp64" (plain FP64 factorizations) or "mixed" (LU and least
    squares: 4-digit tensor-core updates + FP64 refinement)."""

    def __init__(self, hbm_budget: int, slots: int = 4, b: int = 128, leaf_rows: int = 256,
                 levels=((4, 0), (0, 0)), form: str = "fp64", device: int = 0, execute=None):
        self.budget = int(hbm_budget)
        self.b = b
        self.leaf_rows = leaf_rows
        self.levels = tuple(levels)
        self.form = form
        self.device = device
        self._on_gpu = execute is None
        self._execute = execute or self._run_on_gpu
        self._pending: queue.Queue = queue.Queue()
        self._cv = threading.Condition()
        self._used = 0
        self._running = 0
        self.max_running = 0
        self._free_slots = list(range(slots))
        self._work = [queue.Queue() for _ in range(slots)]
        self.max_used = 0
        self._submitted = 0
        self._finished = 0
        self.completed: list[Request] = []
        self.rejected: list[Request] = []
        self.cancelled: list[Request] = []
        self._stop = False
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        self._sched.start()
        for w in self._workers:
            w.start()

    # ---- public ------------------------------------------------------------
    def tree(self):
        lv = self.levels
        return B.make_tree(self.leaf_rows, lv)

    def submit(self, kind: str, A: np.ndarray, Bm: np.ndarray) -> Request:
        if Bm.ndim == 1:
            Bm = Bm[:, None]
        r = Request(kind, np.asfortranarray(A), np.asfortranarray(Bm), arrival=time.perf_counter())
        m, n = r.A.shape
        if kind == LU and m != n:
            raise ValueError("lu requests need a square matrix")
        if kind == LS and m < n:
            raise ValueError("ls requests need m >= n")
        r.footprint = footprint(kind, m, n, r.B.shape[1], self.b, self.tree(), self.form)
        with self._cv:
            self._submitted += 1
        self._pending.put(r)
        return r

    def cancel(self, r: Request) -> bool:
        """Withdraws a request that has not started: True if it was still
        pending (it finishes as "cancelled" and nothing of it reaches the GPU),
        False if it already runs or has finished.  A running request is never
        interrupted: its kernels complete and its result is kept."""
        with self._cv:
            if r.status != "pending":
                return False
            r.status = "cancelled"
            r.t_done = time.perf_counter()
            self.cancelled.append(r)
            self._finish(r)
            return True

    def _finish(self, r: Request):
        with self._cv:
            self._finished += 1
            self._cv.notify_all()
        r.done.set()

    def drain(self, timeout: float = 600.0):
        """Wait until every submitted request is done, failed, rejected or
        cancelled."""
        deadline = time.perf_counter() + timeout
        with self._cv:
            while self._finished < self._submitted:
                left = deadline - time.perf_counter()
                if left <= 0:
                    raise TimeoutError("requests still pending")
                self._cv.wait(timeout=min(left, 0.05))

    def close(self):
        self._stop = True
        self._pending.put(None)
        for q in self._work:
            q.put(None)
        self._sched.join(timeout=10)
        for w in self._workers:
            w.join(timeout=10)

    def stats(self) -> dict:
        out = latency_stats(self.completed)
        out.update({"rejected": len(self.rejected), "cancelled": len(self.cancelled)})
        if self.completed:
            out.update({"max_hbm_in_use": self.max_used, "budget": self.budget,
                        "max_running": self.max_running, "max_on_device": self.max_on_device()})
        return out

    def max_on_device(self) -> int:
        """Most requests whose device intervals (CUDA events on their streams)
        overlapped at one instant: > 1 means their kernels ran concurrently."""
        return max_overlap(self.completed)

    # ---- scheduler: admission by HBM footprint, arrival order ---------------
    def _schedule(self):
        while not self._stop:
            r = self._pending.get()
            if r is None:
                return
            with self._cv:
                if r.status == "cancelled":  # finished by cancel()
                    continue
                if r.footprint > self.budget:
                    r.status = "rejected"
                    r.t_done = time.perf_counter()
                    self.rejected.append(r)
                    self._finish(r)
                    continue
                # arrival order: the head request waits for a slot and memory
                while not self._stop and r.status != "cancelled" and (
                        not self._free_slots or self._used + r.footprint > self.budget):
                    self._cv.wait(timeout=0.05)
                if self._stop:
                    return
                if r.status == "cancelled":
                    continue
                slot = self._free_slots.pop(0)
                self._used += r.footprint
                self.max_used = max(self.max_used, self._used)
                self._running += 1
                self.max_running = max(self.max_running, self._running)
                r.status = "running"
            self._work[slot].put(r)

    def _release(self, slot: int, r: Request):
        with self._cv:
            self._used -= r.footprint
            self._running -= 1
            self._free_slots.append(slot)
            self._cv.notify_all()

    def _worker(self, slot: int):
        ctx = None
        while True:
            r = self._work[slot].get()
            if r is None:
                return
            try:
                if ctx is None:
                    ctx = self._make_context()
                r.X = self._execute(r, ctx)
                r.status = "done"
            except Exception as e:  # the request fails, the server keeps serving
                r.status = "failed"
                r.error = repr(e)
            r.t_done = time.perf_counter()
            if r.status == "done":
                self.completed.append(r)
            self._release(slot, r)
            self._finish(r)

    # ---- execution on the GPU -------------------------------------------------
    def _make_context(self):
        if not self._on_gpu:
            return None
        import torch
        torch.cuda.set_device(self.device)
        with self._cv:
            if not hasattr(self, "_ref_event"):
                # reference instant of the device intervals (recorded once, before any request)
                self._ref_event = torch.cuda.Event(enable_timing=True)
                self._ref_event.record(torch.cuda.current_stream(self.device))
                self._ref_event.synchronize()
        return torch.cuda.Stream(device=self.device)

    def _run_on_gpu(self, r: Request, stream):
        return solve_request(r, stream, self.form, self.b, self.tree(), self.device, self._ref_event)


def latency_stats(completed) -> dict:
    """p50 / p99 latency (arrival to result on the host) and goodput (completed
    requests over the span from the first arrival to the last result)."""
    lat = sorted(r.latency for r in completed)
    if not lat:
        return {"completed": 0}
    pct = lambda p: lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)]
    span = max(r.t_done for r in completed) - min(r.arrival for r in completed)
    return {"completed": len(lat), "p50_s": pct(0.50), "p99_s": pct(0.99),
            "solves_per_s": len(lat) / span if span > 0 else float("inf")}


def max_overlap(completed) -> int:
    """Most requests whose device intervals (gpu_ms) overlap at one instant."""
    ev = []
    for r in completed:
        if r.gpu_ms:
            ev.append((r.gpu_ms[0], 1))
            ev.append((r.gpu_ms[1], -1))
    ev.sort(key=lambda e: (e[0], e[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def solve_request(r: Request, stream, form: str, b: int, tree, device: int, ref_event=None):
    """One request on `stream` through the C-ABI: the matrix and right-hand
    sides to the device, the factorization and solve of the form ("fp64":
    calu_factor + calu_getrs / caqr_factor + caqr_geqrs; "mixed": LU by
    calu_gesv_mixed with 4 digits and automatic refinement, least squares by
    caqr_gels_mixed with 4 digits and refinement), the solution back to the
    host.  Raises when the library reports a problem (check_result)."""
    import torch
    dev = torch.device("cuda", device)
    m, n = r.A.shape
    nrhs = r.B.shape[1]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    berr = None
    with torch.cuda.stream(stream):
        t0.record(stream)
        A = torch.from_numpy(np.ascontiguousarray(r.A.T)).to(dev, non_blocking=True).t()
        Bm = torch.from_numpy(np.ascontiguousarray(r.B.T)).to(dev, non_blocking=True).t()
        swork = None
        if r.kind == LU and form == "mixed":
            X, it, berr, info = B.calu_gesv_mixed(A, Bm, b, tree, slices=4, exact=True, tol=1e-14,
                                                  refine="auto", stream=stream)
        elif r.kind == LU:
            ipiv, info = B.calu_factor(A, b, tree, stream=stream)
            swork = B._buf(B.ca_getrs_workspace(n, nrhs), dev)
            B.calu_getrs(A, ipiv, Bm, work=swork, stream=stream)
            X = Bm
        elif form == "mixed":
            X, it, berr, info = B.caqr_gels_mixed(A, Bm, b, tree, slices=4, exact=True, max_iter=10, tol=1e-14,
                                                  stream=stream)
        else:
            qtree, info = B.caqr_factor(A, b, tree, stream=stream)
            swork = B._buf(B.ca_geqrs_workspace(m, n, nrhs, b, tree), dev)
            B.caqr_geqrs(A, b, tree, qtree, Bm, work=swork, stream=stream)
            X = Bm[:n]
        out = X.cpu()  # waits for this request's stream only
        t1.record(stream)
        stream.synchronize()
    if ref_event is not None:
        r.gpu_ms = (ref_event.elapsed_time(t0), ref_event.elapsed_time(t1))
    check_result(info.cpu().tolist(), B.ca_solve_status(swork, stream) if swork is not None else False,
                 None if berr is None else float(berr.item()))
    if berr is not None:
        r.berr = float(berr.item())
    return np.asfortranarray(out.numpy())


def run_plain(items, form: str = "fp64", b: int = 128, leaf_rows: int = 256, levels=((4, 0), (0, 0)),
              device: int = 0):
    """The plain per-request form the server is compared with: one thread, one
    stream, requests taken in arrival order as they arrive (no admission, no
    overlap), each solved to completion before the next starts.  items:
    (arrival in seconds after the start, kind, A, B).  Returns the requests
    with their results and latencies."""
    import torch
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device=device)
    tree = B.make_tree(leaf_rows, levels)
    done = []
    t_start = time.perf_counter()
    for t_arr, kind, A, Bm in items:
        now = time.perf_counter() - t_start
        if t_arr > now:
            time.sleep(t_arr - now)
        if Bm.ndim == 1:
            Bm = Bm[:, None]
        r = Request(kind, np.asfortranarray(A), np.asfortranarray(Bm), arrival=t_start + t_arr)
        r.status = "running"
        try:
            r.X = solve_request(r, stream, form, b, tree, device)
            r.status = "done"
        except Exception as e:  # noqa: BLE001 -- the request fails, the loop goes on
            r.status = "failed"
            r.error = repr(e)
        r.t_done = time.perf_counter()
        r.done.set()
        done.append(r)
    return done


def check_result(info, solve_timed_out: bool, berr=None):
    """Raises (the request fails) when the library reported a problem: a zero
    pivot (info[0]), a NaN / Inf in a panel or a tensor-core or solve timeout
    (info[1]), a triangular solve that gave up waiting, or a refinement that
    ended with a non-finite backward error."""
    if info[0] != 0:
        raise RuntimeError(f"U({info[0] - 1}, {info[0] - 1}) is exactly zero: the matrix is singular")
    if info[1] != 0:
        raise RuntimeError(f"status bits {info[1]:#x} (1: NaN/Inf in a panel, 2/4/8: tensor-core wait "
                           "timeout, 16: triangular-solve wait timeout)")
    if solve_timed_out:
        raise RuntimeError("a triangular solve gave up waiting for a block (result only partly solved)")
    if berr is not None and not math.isfinite(berr):
        raise RuntimeError(f"refinement ended with backward error {berr}")


def poisson_workload(rate: float, duration: float, seed: int, nmin: int = 64, nmax: int = 2048,
                     ls_fraction: float = 0.5, max_rhs: int = 16, count: int | None = None, sizes=None):
    """Arrival times and shapes of an open-loop Poisson stream: n log-uniform in
    [nmin, nmax] (snapped to the nearest of `sizes` in log scale, when given),
    LU (m = n) or LS (m = 4n) requests, 1..max_rhs right-hand sides; the
    arrivals of `duration` seconds, or the first `count` arrivals."""
    g = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if (count is None and t > duration) or (count is not None and len(out) >= count):
            return out
        n = int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax)))))
        if sizes:
            n = min(sizes, key=lambda s_: abs(math.log(s_) - math.log(n)))
        kind = LS if g.uniform() < ls_fraction else LU
        m = 4 * n if kind == LS else n
        out.append((t, kind, m, n, int(g.integers(1, max_rhs + 1))))
