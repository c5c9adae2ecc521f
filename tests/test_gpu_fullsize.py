"""GPU parity at the full sizes of the workloads, in the configurations the
benchmark times.

Where the oracle finishes in seconds it runs in full (tall-skinny TSLU / TSQR
panels of 1,048,576 x 64 and 8,388,608 x 32 with 256-row leaves: pivots must
match exactly, factors, every stored Y and every T within 1e-12).  At
n = 16384 (b = 128, the benchmark's leaves and tree) the oracle computes
the first panel's tournament exactly and sampled outputs one by one: rows of
P A - L U, column norms of R, backward errors of the solves, and the tensor-core
forms against the FP64 form.
"""
import numpy as np
import pytest

import bench
import oracle
from paper_1303_5837_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TREE4 = [(4, 0), (8, 0), (0, 0)]   # leaves in groups of 4, then 8, then the grid
BENCH_TREE = bench.parse_tree(bench.BENCH_TREE)


@pytest.fixture(scope="module")
def ca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1303_5837_gb300 as ca
    ca.load()
    return ca


def to_dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).cuda().t()


def rows_from_ipiv(ipiv, m):
    perm = np.arange(m)
    for i, p in enumerate(ipiv):
        p -= 1
        perm[i], perm[p] = perm[p], perm[i]
    return perm


@pytest.mark.parametrize("m,n", [(1_048_576, 64), (8_388_608, 32)])
def test_tslu_full_size(ca, m, n):
    L = 256
    A = inputs.gaussian(m, n, 2026)
    sel, nt = oracle.tslu_select(A, oracle.make_tree(L, TREE4))
    assert nt == 0
    Ad = to_dev(A)
    ipiv, info = ca.tslu(Ad, ca.make_tree(L, TREE4))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    perm = rows_from_ipiv(ipiv.cpu().numpy(), m)
    assert np.array_equal(perm[:n], sel)
    # U11 and L11: the LU without pivoting of the selected rows
    LU = Ad[:n].cpu().numpy()
    S = A[sel].copy()
    for j in range(n):
        S[j + 1:, j] /= S[j, j]
        S[j + 1:, j + 1:] -= np.outer(S[j + 1:, j], S[j, j + 1:])
    assert np.linalg.norm(LU - S) / np.linalg.norm(S) < 1e-12
    # sampled rows of L21 = A21 U11^-1
    rng = np.random.default_rng(1)
    rows = rng.choice(np.arange(n, m), 2000, replace=False)
    U = np.triu(S)
    want = np.linalg.solve(U.T, A[perm[rows]].T).T
    got = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


@pytest.mark.parametrize("m,n", [(1_048_576, 64), (8_388_608, 32)])
def test_tsqr_full_size(ca, m, n):
    L = 256
    A = inputs.gaussian(m, n, 2027)
    QR_o, T_o = oracle.tsqr(A, oracle.make_tree(L, TREE4))
    Ad = to_dev(A)
    qtree, info = ca.tsqr(Ad, ca.make_tree(L, TREE4))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    QR = Ad.cpu().numpy()
    R, R_o = np.triu(QR[:n]), np.triu(QR_o[:n])
    assert np.linalg.norm(R - R_o) / np.linalg.norm(R_o) < 1e-12
    assert np.linalg.norm(QR - QR_o) / np.linalg.norm(QR_o) < 1e-12      # every stored Y
    T = qtree.cpu().numpy()[: T_o.size]
    assert np.linalg.norm(T - T_o) / np.linalg.norm(T_o) < 1e-12          # every T


@pytest.fixture(scope="module")
def big():
    """The benchmark's matrix family at n = 16384 (cond 1e6), on the device."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    n = 16384
    A0 = bench.conditioned_device(n, 1e6, 2026, torch.device("cuda", 0))
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(n, 1, dtype=torch.float64, device="cuda", generator=g)
    B0 = (A0 @ x).t().contiguous().t()
    return A0, B0, x


def berr(A, X, B):
    R = B - A @ X
    return float((R.abs().amax(0) / (A.abs().sum(1).amax() * X.abs().amax(0) + B.abs().amax(0))).max())


def lu_rows_residual(LU, perm, A0, count=48, seed=3):
    """|| (P A - L U)(rows, :) || / || (P A)(rows, :) || for sampled rows."""
    n = A0.shape[0]
    rows = np.random.default_rng(seed).choice(n, count, replace=False)
    rt = torch.from_numpy(rows).cuda()
    below = torch.arange(n, device="cuda")[None, :] < rt[:, None]
    Lr = torch.where(below, LU[rt], torch.zeros((), dtype=LU.dtype, device="cuda"))
    Lr[torch.arange(count, device="cuda"), rt] = 1.0
    LUr = Lr @ torch.triu(LU)
    PAr = A0[torch.from_numpy(perm[rows]).cuda()]
    return float(torch.linalg.norm(LUr - PAr) / torch.linalg.norm(PAr))


def test_calu_bench_configuration(ca, big):
    A0, B0, x = big
    import bench
    n, b, L = A0.shape[0], 128, bench.BENCH_LEAF_ROWS
    tree = ca.make_tree(L, BENCH_TREE)
    # first panel: the tournament over 64 leaves, exactly the oracle's
    P = A0[:, :b].cpu().numpy()
    sel, nt = oracle.tslu_select(P, oracle.make_tree(L, BENCH_TREE))
    assert nt == 0
    A = A0.clone()
    ipiv, info = ca.calu_factor(A, b, tree)
    X = B0.clone()
    ca.calu_getrs(A, ipiv, X)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    perm = rows_from_ipiv(ipiv.cpu().numpy(), n)
    assert np.array_equal(perm[:b], sel)
    assert lu_rows_residual(A, perm, A0) < 1e-13
    assert berr(A0, X, B0) < 1e-15
    # the tensor-core forms.  (At cond 1e6 two backward-stable factorizations
    # differ elementwise in the late, ill-conditioned panels, so the FP64-level
    # agreement of the 7-digit form is pinned on well-conditioned inputs in
    # test_gpu_mixed.py; here: same pivots, same backward errors.)
    A7 = A0.clone()
    ipiv7, info7 = ca.calu_factor_mixed(A7, b, tree, slices=7, exact=True)
    X7 = B0.clone()
    ca.calu_getrs(A7, ipiv7, X7)
    torch.cuda.synchronize()
    assert torch.equal(ipiv7, ipiv)
    assert lu_rows_residual(A7, perm, A0) < 1e-13
    assert berr(A0, X7, B0) < 1e-15
    Xm, iters, be, infom = ca.calu_gesv_mixed(A0, B0, b, tree, slices=4, exact=True, tol=1e-14)
    torch.cuda.synchronize()
    assert be <= 1e-14 and berr(A0, Xm, B0) < 1e-14
    # forward errors: kappa_2 (1e6) times the backward error, with a factor
    # sqrt(n) between the infinity-norm backward error and the 2-norm bound
    fwd = lambda Y: float(torch.linalg.norm(Y - x) / torch.linalg.norm(x))
    bound = 1e6 * 1e-14 * np.sqrt(n)
    assert fwd(X) < bound and fwd(X7) < bound and fwd(Xm) < bound


def test_caqr_bench_configuration(ca, big):
    A0, B0, x = big
    import bench
    n, b, L = A0.shape[0], 128, bench.BENCH_LEAF_ROWS
    tree = ca.make_tree(L, BENCH_TREE)
    A = A0.clone()
    qtree, info = ca.caqr_factor(A, b, tree)
    X = B0.clone()
    ca.caqr_geqrs(A, b, tree, qtree, X)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    cols = torch.from_numpy(np.random.default_rng(4).choice(n, 64, replace=False)).cuda()

    def colnorm_err(QR):
        # sampled columns: ||R(:, j)|| = ||A(:, j)|| (Q is orthogonal)
        nr = torch.linalg.norm(torch.triu(QR)[:, cols], dim=0)
        na = torch.linalg.norm(A0[:, cols], dim=0)
        return float(((nr - na).abs() / na).max())

    assert colnorm_err(A) < 1e-13
    assert berr(A0, X, B0) < 1e-14
    A7 = A0.clone()
    q7, _ = ca.caqr_factor_mixed(A7, b, tree, slices=7, exact=True)
    X7 = B0.clone()
    ca.caqr_geqrs(A7, b, tree, q7, X7)
    torch.cuda.synchronize()
    assert colnorm_err(A7) < 1e-13
    assert berr(A0, X7, B0) < 1e-14
    # the first panel is well determined: its R rows agree to FP64 level
    assert float(torch.linalg.norm(torch.triu(A7[:b]) - torch.triu(A[:b])) / torch.linalg.norm(torch.triu(A[:b]))) < 1e-12
