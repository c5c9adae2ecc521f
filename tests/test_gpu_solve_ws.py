"""The solves keep their synchronization state in caller memory and report a
wait that runs out (GPU).

* calu_getrs, caqr_geqrs and calu_gesv_mixed allocate no device memory, also
  on the first call on a new stream: the ready flags of the dependency-ordered
  triangular solves live in the workspace the caller passes.
* A wait on a ready flag that nothing sets gives up after its limit: the test
  hook withholds the first block's flag, the solve returns, the timeout is
  reported (ca_solve_status for calu_getrs / caqr_geqrs, a dev_info bit for
  calu_gesv_mixed), and the next solve on the same stream is correct again.
"""
import numpy as np
import pytest

from paper_1303_5837_gb300 import inputs


def berr(A, X, B):
    """Largest normwise backward error ||b - A x||inf / (||A||inf ||x||inf + ||b||inf)."""
    R = B - A @ X
    return float((np.abs(R).max(0) / (np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0))).max())

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHORT_WAIT = 2_000_000   # SM clock cycles, about 1 ms


@pytest.fixture(scope="module")
def ca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1303_5837_gb300 as ca
    ca.load()
    return ca


def to_dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).cuda().t()


@pytest.fixture(scope="module")
def lu_case(ca):
    n, b, L = 1536, 128, 256
    A = inputs.gaussian(n, n, 61)
    B = inputs.rhs(n, 2, 62)
    t = ca.make_tree(L)
    LU = to_dev(A)
    ipiv, info = ca.calu_factor(LU, b, t)
    torch.cuda.synchronize()
    return A, B, LU, ipiv, None


def test_solves_allocate_nothing_on_a_new_stream(ca, lu_case):
    A, B, LU, ipiv, x_o = lu_case
    n = A.shape[0]
    work = torch.zeros((ca.ca_getrs_workspace(n, 2) + 7) // 8, dtype=torch.float64, device="cuda")
    X = to_dev(B)
    ca.calu_getrs(LU, ipiv, X, work=work)          # kernels loaded, attributes set
    m, nq, b, L = 3000, 700, 64, 256
    t = ca.make_tree(L)
    Aq = to_dev(inputs.gaussian(m, nq, 63))
    qtree, _ = ca.caqr_factor(Aq, b, t)
    qwork = torch.zeros((ca.ca_geqrs_workspace(m, nq, 1, b, t) + 7) // 8, dtype=torch.float64, device="cuda")
    Bq = to_dev(inputs.rhs(m, 1, 64))
    Bq0 = Bq.clone()
    ca.caqr_geqrs(Aq, b, t, qtree, Bq, work=qwork)
    torch.cuda.synchronize()
    for _ in range(3):
        s = torch.cuda.Stream()
        X2 = to_dev(B)
        Bq.copy_(Bq0)
        torch.cuda.synchronize()
        before, _ = torch.cuda.mem_get_info()
        ca.calu_getrs(LU, ipiv, X2, work=work, stream=s)
        ca.caqr_geqrs(Aq, b, t, qtree, Bq, work=qwork, stream=s)
        s.synchronize()
        after, _ = torch.cuda.mem_get_info()
        assert after == before, (before - after)
        assert berr(A, X2.cpu().numpy(), B) < 1e-14


def test_flag_wait_runs_out_and_is_reported(ca, lu_case):
    A, B, LU, ipiv, x_o = lu_case
    n = A.shape[0]
    work = torch.zeros((ca.ca_getrs_workspace(n, 2) + 7) // 8, dtype=torch.float64, device="cuda")
    X = to_dev(B)
    ca.ca_test_solve_hook(SHORT_WAIT, True)
    try:
        ca.calu_getrs(LU, ipiv, X, work=work)
        assert ca.ca_solve_status(work) is True       # the waits gave up and said so
    finally:
        ca.ca_test_solve_hook(0, False)
    # the stream and the context stay usable: the same solve is right again
    X = to_dev(B)
    ca.calu_getrs(LU, ipiv, X, work=work)
    assert ca.ca_solve_status(work) is False
    assert berr(A, X.cpu().numpy(), B) < 1e-14


def test_flag_wait_runs_out_in_geqrs_and_refinement(ca):
    m, n, b, L = 2000, 600, 64, 256
    t = ca.make_tree(L)
    A = to_dev(inputs.gaussian(m, n, 71))
    qtree, _ = ca.caqr_factor(A, b, t)
    Bq = to_dev(inputs.rhs(m, 1, 72))
    work = torch.zeros((ca.ca_geqrs_workspace(m, n, 1, b, t) + 7) // 8, dtype=torch.float64, device="cuda")
    As = inputs.conditioned(1024, 1e4, 73)
    Bs = As @ inputs.rhs(1024, 1, 74)
    ca.ca_test_solve_hook(SHORT_WAIT, True)
    try:
        ca.caqr_geqrs(A, b, t, qtree, Bq.clone(), work=work)
        assert ca.ca_solve_status(work) is True
        _, _, _, info = ca.calu_gesv_mixed(to_dev(As), to_dev(Bs), 128, ca.make_tree(256), slices=4,
                                           exact=True, max_iter=3)
        torch.cuda.synchronize()
        assert info.cpu().tolist()[1] & ca.CA_STATUS_SOLVE_TIMEOUT
    finally:
        ca.ca_test_solve_hook(0, False)
    ca.caqr_geqrs(A, b, t, qtree, Bq.clone(), work=work)
    assert ca.ca_solve_status(work) is False
    X, it, be, info = ca.calu_gesv_mixed(to_dev(As), to_dev(Bs), 128, ca.make_tree(256), slices=4, exact=True)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0] and float(be.item()) <= 1e-14
