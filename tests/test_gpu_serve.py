"""The serving loop on the GPU: a mix of LU and least-squares requests of
uneven sizes runs concurrently on several streams; every result equals the
same request solved alone (the kernels are deterministic, so exactly), and
matches the CPU oracle."""
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
