"""The serving loop on the GPU: a mix of LU and least-squares requests of
uneven sizes runs concurrently on several streams -- requests admitted
while others run overlap on the device (their CUDA-event intervals
intersect) -- every result equals the same request solved alone (the
kernels are deterministic, so exactly), and matches the CPU oracle; the
plain per-request loop gives the same answers."""
import numpy as np
import pytest

import oracle
from paper_1303_5837_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_5837_gb300 import serve
    serve.B.load()
    return serve


def make_requests(seed):
    g = np.random.default_rng(seed)
    reqs = []
    for i in range(24):
        n = int(g.choice([64, 100, 256, 333, 512, 777, 1024]))
        kind = "ls" if i % 2 else "lu"
        m = 4 * n if kind == "ls" else n
        nrhs = int(g.integers(1, 5))
        reqs.append((kind, inputs.gaussian(m, n, 100 + i), inputs.gaussian(m, nrhs, 200 + i)))
    return reqs


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_results_same_alone_and_in_the_mix(serve, form):
    reqs = make_requests(1)
    alone = serve.SolveServer(hbm_budget=1 << 34, slots=1, form=form)
    try:
        ref = []
        for kind, A, Bm in reqs:
            r = alone.submit(kind, A, Bm)
            r.done.wait(120)
            ref.append(r.X)
    finally:
        alone.close()
    mix = serve.SolveServer(hbm_budget=1 << 34, slots=4, form=form)
    try:
        got = [mix.submit(kind, A, Bm) for kind, A, Bm in reqs]
        mix.drain(timeout=300)
        st = mix.stats()
    finally:
        mix.close()
    assert st["completed"] == len(reqs), [r.error for r in got if r.status != "done"][:3]
    # continuous batching, not a queue: requests ran on the device at the same time
    assert st["max_running"] >= 2 and st["max_on_device"] >= 2, st
    for r, x in zip(got, ref):
        assert r.status == "done", r.error
        assert np.array_equal(r.X, x)
    # and the answers are the oracle's (FP64 form) / backward stable (mixed)
    for (kind, A, Bm), x in zip(reqs[:6], ref[:6]):
        if kind == "lu":
            LU, ipiv, _, _ = oracle.calu(A, 128, oracle.make_tree(256, [(4, 0), (0, 0)]))
            xo = oracle.getrs(LU, ipiv, Bm)
        else:
            QR, T = oracle.caqr(A, 128, oracle.make_tree(256, [(4, 0), (0, 0)]))
            xo = oracle.geqrs(QR, T, 128, oracle.make_tree(256, [(4, 0), (0, 0)]), Bm)
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-10


def test_plain_loop_matches_the_server(serve):
    """The plain per-request form (one stream, in arrival order, no admission)
    that the server is measured against gives the same answers."""
    reqs = make_requests(2)[:8]
    srv = serve.SolveServer(hbm_budget=1 << 34, slots=1, form="fp64")
    try:
        ref = []
        for kind, A, Bm in reqs:
            r = srv.submit(kind, A, Bm)
            r.done.wait(120)
            ref.append(r.X)
    finally:
        srv.close()
    done = serve.run_plain([(0.0, kind, A, Bm) for kind, A, Bm in reqs], form="fp64")
    assert all(r.status == "done" for r in done), [r.error for r in done]
    for r, x in zip(done, ref):
        assert np.array_equal(r.X, x)
