"""GPU tests of the reduced-precision path: the tcgen05 digit-split update,
the mixed CALU and FP64 iterative refinement.

The update is checked against the plain definition C - A B in FP64 (numpy),
with the error bound of its digit count; exact mode on integer digits must be
bit-exact (the tensor cores' FP32 sums of integers below 2^24 are exact).
The mixed factorizations are checked against the CPU oracle: with 7 exact
digits the update is FP64-accurate and the pivots must equal the oracle's;
refinement must reach a backward error <= 1e-14 and the oracle's solution.
"""
import numpy as np
import pytest

import oracle
from paper_1303_5837_gb300 import inputs
from tests.parity import check, lu_err, qr_err, qtree_err, solve_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1303_5837_gb300 as ca
    ca.load()
    return ca


def to_dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).cuda().t()


def to_host(T):
    return np.asfortranarray(T.cpu().numpy())


def scaled_err(C_gpu, C_ref, A, B):
    """max |error| over max_i max|A(i,:)| max_j max|B(:,j)| k."""
    k = A.shape[1]
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * k
    return float(np.max(np.abs(C_gpu - C_ref) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (300, 200, 128), (1000, 700, 100), (513, 257, 128),
                                   (129, 1000, 32), (4096, 4096, 128)])
@pytest.mark.parametrize("slices,exact,bound", [(2, False, 2.0 ** -14), (3, False, 2.0 ** -18),
                                                (3, True, 2.0 ** -22), (4, True, 2.0 ** -30),
                                                (6, True, 2.0 ** -44), (7, True, 2.0 ** -50)])
def test_gemm_mixed_accuracy(ca, m, n, k, slices, exact, bound):
    A = inputs.gaussian(m, k, m + k)
    B = inputs.gaussian(k, n, n + k) * 10.0
    C = inputs.gaussian(m, n, m + n)
    Cd = to_dev(C)
    st = ca.ca_gemm_minus_mixed(to_dev(A), to_dev(B), Cd, slices=slices, exact=exact)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = C - A @ B
    assert scaled_err(to_host(Cd), ref, A, B) < bound


def test_gemm_exact_mode_is_exact_on_integers(ca):
    """Integer operands below 256 are single digits: the exact mode must give
    C - A B with no rounding at all (FP32 sums of integers < 2^24 on the
    tensor cores, FP64 epilogue)."""
    m, n, k = 384, 256, 128
    A = inputs.int_matrix(m, k, 1, -255, 255)
    B = inputs.int_matrix(k, n, 2, -255, 255)
    C = inputs.int_matrix(m, n, 3, -1000, 1000)
    Cd = to_dev(C)
    ca.ca_gemm_minus_mixed(to_dev(A), to_dev(B), Cd, slices=1, exact=True)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(Cd), C - A @ B)


@pytest.mark.parametrize("m,n,b,L", [(1024, 1024, 64, 128), (777, 500, 48, 96), (1500, 1500, 128, 256)])
def test_calu_mixed_exact7_matches_oracle(ca, m, n, b, L):
    A = inputs.gaussian(m, n, 3 * m + n)
    tree = [(2, 0), (0, 0)]
    LU_o, ipiv_o, _, nt = oracle.calu(A, b, oracle.make_tree(L, tree))
    assert nt == 0
    Ad = to_dev(A)
    ipiv, info = ca.calu_factor_mixed(Ad, b, ca.make_tree(L, tree), slices=7, exact=True)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_o)
    check(lu_err(to_host(Ad), LU_o), 1e-12, (m, n, b))


def test_calu_mixed_fused_backward_error(ca):
    n, b, L = 2048, 128, 256
    A = inputs.gaussian(n, n, 99)
    Ad = to_dev(A)
    ipiv, info = ca.calu_factor_mixed(Ad, b, ca.make_tree(L), slices=3, exact=False)
    torch.cuda.synchronize()
    perm, Lf, U = oracle.lu_unpack(to_host(Ad), ipiv.cpu().numpy())
    res = np.linalg.norm(A[perm] - Lf @ U) / np.linalg.norm(A)
    assert res < 1e-4  # three fused digits: about 2e-5 at n = 2048
    assert info.cpu().tolist() == [0, 0]


@pytest.mark.parametrize("n,cond,slices,exact,nrhs", [(1024, 1e2, 3, False, 2), (1024, 1e6, 3, True, 2),
                                                      (2048, 1e6, 4, True, 2), (1024, 1e10, 5, True, 2),
                                                      (1536, 1e10, 6, True, 2), (2048, 1e6, 4, True, 1),
                                                      (1024, 1e6, 4, True, 6)])
def test_gesv_mixed_refinement(ca, n, cond, slices, exact, nrhs):
    A = inputs.conditioned(n, cond, 7)
    x_true = inputs.rhs(n, nrhs, 8)
    B = A @ x_true
    b, L = 128, 256
    LU_o, ipiv_o, _, _ = oracle.calu(A, b, oracle.make_tree(L))
    x_o = oracle.getrs(LU_o, ipiv_o, B)
    X, iters, berr, info = ca.calu_gesv_mixed(to_dev(A), to_dev(B), b, ca.make_tree(L), slices=slices,
                                              exact=exact, max_iter=30, tol=1e-14)
    torch.cuda.synchronize()
    assert info.cpu().tolist()[1] == 0
    assert float(berr.item()) <= 1e-14, (int(iters.item()), float(berr.item()))
    x = to_host(X)
    # both solutions are backward stable (<= 1e-14): they agree to cond * 1e-14
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) < max(1e-12, cond * 1e-14)


def host_refinement_reference(ca, A, B, b, L, slices, exact, max_iter, tol):
    """The classic refinement loop driven from the host (one wait per step),
    from the same calls: the device-side stop test must take the same steps."""
    n = A.shape[0]
    Ad, Bd = to_dev(A), to_dev(B)
    LU = Ad.clone()
    ipiv, info = ca.calu_factor_mixed(LU, b, ca.make_tree(L), slices=slices, exact=exact)
    X = Bd.clone()
    ca.calu_getrs(LU, ipiv, X)
    anorm = float(Ad.abs().sum(1).amax())
    prev, stall, hist = 0.0, 0, []
    for it in range(max_iter + 1):
        R = Bd - Ad @ X
        be = float((R.abs().amax(0) / (anorm * X.abs().amax(0) + Bd.abs().amax(0))).max())
        hist.append(be)
        if be <= tol or it >= max_iter:
            break
        if it > 0 and be > 0.5 * prev:
            stall += 1
            if stall >= 2:
                break
        else:
            stall = 0
        prev = be
        ca.calu_getrs(LU, ipiv, R)
        X = X + R
    return it, hist


@pytest.mark.parametrize("cond,slices", [(1e6, 3), (1e10, 4)])
def test_device_stop_test_takes_the_host_loops_steps(ca, cond, slices):
    """The stop test runs on the device (the call never waits): it stops at
    the same step as the same loop driven from the host."""
    n, b, L = 1024, 128, 256
    A = inputs.conditioned(n, cond, 11)
    B = A @ inputs.rhs(n, 1, 12)
    it_h, hist = host_refinement_reference(ca, A, B, b, L, slices, True, 12, 1e-14)
    X, iters, berr, info = ca.calu_gesv_mixed(to_dev(A), to_dev(B), b, ca.make_tree(L), slices=slices,
                                              exact=True, max_iter=12, tol=1e-14)
    torch.cuda.synchronize()
    assert int(iters.item()) == it_h, (int(iters.item()), hist)
    assert abs(float(berr.item()) - hist[-1]) <= 1e-3 * hist[-1] + 1e-300


@pytest.mark.parametrize("n,cond,slices,nrhs,max_iter", [(1024, 1e10, 4, 1, 10), (1024, 1e10, 4, 3, 10),
                                                          (4096, 1e6, 3, 1, 6)])
def test_gmres_refinement_where_classic_stalls(ca, n, cond, slices, nrhs, max_iter):
    """GMRES-based refinement (FP64 GMRES on the system preconditioned by the
    reduced-precision factors) reaches backward error 1e-14 with digit counts
    for which the classic correction stalls or is too slow.  The solution
    agrees with the oracle's FP64 CALU solution to cond * 1e-14."""
    A = inputs.conditioned(n, cond, 21)
    B = A @ inputs.rhs(n, nrhs, 22)
    b, L = 128, 256
    t = ca.make_tree(L)
    LU_o, ipiv_o, _, _ = oracle.calu(A, b, oracle.make_tree(L))
    x_o = oracle.getrs(LU_o, ipiv_o, B)
    _, it_c, be_c, _ = ca.calu_gesv_mixed(to_dev(A), to_dev(B), b, t, slices=slices, exact=True,
                                          max_iter=max_iter, tol=1e-14, refine="classic")
    X, it, be, info = ca.calu_gesv_mixed(to_dev(A), to_dev(B), b, t, slices=slices, exact=True,
                                         max_iter=max_iter, tol=1e-14, refine="gmres")
    torch.cuda.synchronize()
    assert float(be_c.item()) > 1e-14, "the classic correction converged: the case does not need GMRES"
    assert info.cpu().tolist() == [0, 0]
    assert float(be.item()) <= 1e-14, (int(it.item()), float(be.item()))
    x = to_host(X)
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) < cond * 1e-14


@pytest.mark.parametrize("n,cond,slices,expect", [(1024, 1e6, 4, "classic"), (1024, 1e10, 4, "gmres"),
                                                  (4096, 1e6, 3, "gmres"), (2048, 1e10, 4, "refactor"),
                                                  (1536, 1e8, 3, "refactor")])
def test_auto_refinement_reaches_tol(ca, n, cond, slices, expect):
    """refine="auto": classic corrections, GMRES where they are slow, a
    refactorization with 7 exact digits where GMRES stalls too (reported by
    CA_STATUS_REFACTORED); every case reaches backward error 1e-14 and the
    oracle's solution to cond * 1e-14."""
    A = inputs.conditioned(n, cond, 21)
    B = A @ inputs.rhs(n, 1, 22)
    b, L = 128, 256
    LU_o, ipiv_o, _, _ = oracle.calu(A, b, oracle.make_tree(L))
    x_o = oracle.getrs(LU_o, ipiv_o, B)
    X, it, be, info = ca.calu_gesv_mixed(to_dev(A), to_dev(B), b, ca.make_tree(L), slices=slices, exact=True,
                                         max_iter=10, tol=1e-14, refine="auto")
    torch.cuda.synchronize()
    inf = info.cpu().tolist()
    assert inf[0] == 0 and (inf[1] & ~ca.CA_STATUS_REFACTORED) == 0, inf
    assert bool(inf[1] & ca.CA_STATUS_REFACTORED) == (expect == "refactor"), (inf, expect)
    assert float(be.item()) <= 1e-14, (int(it.item()), float(be.item()), expect)
    x = to_host(X)
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) < max(1e-12, cond * 1e-14)


CAQR_CASES = [
    (1024, 1024, 64, 128, [(0, 0)]),
    (1200, 700, 64, 128, [(2, 0), (0, 0)]),
    (640, 256, 128, 256, [(0, 0)]),
    (900, 333, 32, 100, [(4, 0), (0, 1)]),
    (1000, 300, 48, 96, [(3, 1), (0, 0)]),
]


@pytest.mark.parametrize("m,n,b,L,tree", CAQR_CASES)
def test_caqr_mixed_exact7_matches_oracle(ca, m, n, b, L, tree):
    """The tree update on the tensor cores with 7 exact digits reproduces the
    FP64 oracle's factors, every stored Y and every T element to 1e-12 of its
    rounding scale."""
    A = inputs.gaussian(m, n, 17 + m + n)
    QR_o, T_o = oracle.caqr(A, b, oracle.make_tree(L, tree))
    Ad = to_dev(A)
    qtree, info = ca.caqr_factor_mixed(Ad, b, ca.make_tree(L, tree), slices=7, exact=True)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    t = oracle.make_tree(L, tree)
    check(qr_err(to_host(Ad), QR_o, b), 1e-12, (m, n, b))
    check(qtree_err(qtree.cpu().numpy(), T_o, QR_o, b, t, oracle.tree_counts), 1e-12, (m, n, b))


def test_caqr_mixed_fused_r(ca):
    m, n, b, L = 2048, 1024, 128, 256
    A = inputs.gaussian(m, n, 5)
    Ad = to_dev(A)
    ca.caqr_factor_mixed(Ad, b, ca.make_tree(L), slices=3, exact=False)
    torch.cuda.synchronize()
    R = np.triu(to_host(Ad)[:n])
    Rl = np.linalg.qr(A, mode="r")
    d = np.sign(np.diag(R)) * np.sign(np.diag(Rl))
    assert np.linalg.norm(d[:, None] * R - Rl) / np.linalg.norm(Rl) < 1e-4


def test_caqr_mixed_geqrs(ca):
    """Least squares on the emulated factors equals the oracle's."""
    m, n, b, L = 1500, 400, 64, 128
    tree = [(2, 0), (0, 0)]
    A = inputs.gaussian(m, n, 31)
    B = inputs.rhs(m, 3, 32)
    QR_o, T_o = oracle.caqr(A, b, oracle.make_tree(L, tree))
    x_o = oracle.geqrs(QR_o, T_o, b, oracle.make_tree(L, tree), B)
    Ad = to_dev(A)
    t = ca.make_tree(L, tree)
    qtree, _ = ca.caqr_factor_mixed(Ad, b, t, slices=7, exact=True)
    Bd = to_dev(B)
    ca.caqr_geqrs(Ad, b, t, qtree, Bd)
    torch.cuda.synchronize()
    check(solve_err(to_host(Bd)[:n], x_o), 1e-12)


@pytest.mark.parametrize("m,n,cond,slices,noise,nrhs", [(2048, 512, 1e4, 4, 0.0, 2), (2048, 512, 1e4, 4, 1e-3, 2),
                                                        (3000, 700, 1e6, 4, 1e-6, 2), (1500, 400, 1e2, 3, 1e-2, 2),
                                                        (2048, 512, 1e6, 4, 1e-3, 1), (1700, 600, 1e4, 4, 0.0, 5)])
def test_gels_mixed_refinement(ca, m, n, cond, slices, noise, nrhs):
    """Least squares after a reduced-digit CAQR, refined on the corrected
    semi-normal equations: the stop measure (||A^T r|| over its scale)
    reaches 1e-14 and the solution is the oracle's FP64 CAQR least-squares
    solution within the sensitivity of the problem (cond eps, plus
    cond^2 eps ||r|| / (||A|| ||x||) when b is not in the range of A)."""
    g = np.random.default_rng(m + n)
    U, _ = np.linalg.qr(g.standard_normal((m, n)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    s = cond ** (-np.arange(n) / (n - 1))
    A = np.asfortranarray((U * s) @ V.T)
    x_true = g.standard_normal((n, nrhs))
    e = g.standard_normal((m, nrhs))
    e -= U @ (U.T @ e)                             # orthogonal to range(A)
    B = A @ x_true + noise * e / np.linalg.norm(e, axis=0) * np.linalg.norm(A @ x_true, axis=0)
    b, L = 64, 256
    t = oracle.make_tree(L, [(2, 0), (0, 0)])
    QR_o, T_o = oracle.caqr(A, b, t)
    x_o = oracle.geqrs(QR_o, T_o, b, t, B)
    X, it, be, info = ca.caqr_gels_mixed(to_dev(A), to_dev(B), b, ca.make_tree(L, [(2, 0), (0, 0)]),
                                         slices=slices, exact=True, max_iter=10, tol=1e-14)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    assert float(be.item()) <= 1e-14, (int(it.item()), float(be.item()))
    x = to_host(X)
    r = B - A @ x_o
    sens = cond * 1e-15 + cond ** 2 * 1e-16 * np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(x_o))
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) < max(1e-12, 100 * sens)
    # the least-squares condition, in FP64 on the host
    rr = B - A @ x
    assert np.abs(A.T @ rr).max() / (np.abs(A).sum(0).max() * (np.abs(A).sum(1).max() * np.abs(x).max()
                                                               + np.abs(B).max())) < 1e-14
