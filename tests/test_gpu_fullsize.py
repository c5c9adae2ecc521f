"""GPU parity at the full sizes of the workloads, in the configurations the
benchmark times.

Where the oracle finishes in seconds it runs in full, and every element is
compared (``tests/parity.py``):
  * tall-skinny TSLU / TSQR panels of 1,048,576 x 64 and 8,388,608 x 32 with
    256-row leaves: pivots exactly; L, U, R, every stored Y and every T
    element within 1e-12 of its rounding scale;
  * CALU and CAQR of a 4096 x 4096 matrix in the benchmark's own shape
    (b = 128, 1024-row leaves, one flat merge per group of 4 leaves then one
    flat merge of the groups, 32 panels): pivots exactly over all panels,
    every factor, Y and T element.
At n = 16384 (the benchmark's size) the oracle computes the first panel's
tournament exactly and sampled outputs one by one: rows of P A - L U, column
norms of R, backward errors of the solves, and the tensor-core forms against
the FP64 form.
"""
import numpy as np
import pytest

import bench
import oracle
from paper_1303_5837_gb300 import inputs
from tests.parity import check, lu_err, qr_err, qtree_err

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
    t = oracle.make_tree(L, TREE4)
    LU_o, ipiv_o, info_o, nt = oracle.calu(A, n, t, ld_pad=8)
    assert nt == 0 and info_o == 0
    Ad = to_dev(A)
    del A
    ipiv, info = ca.tslu(Ad, ca.make_tree(L, TREE4))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_o)
    check(lu_err(Ad.cpu().numpy(), LU_o), 1e-12, (m, n))


@pytest.mark.parametrize("m,n", [(1_048_576, 64), (8_388_608, 32)])
def test_tsqr_full_size(ca, m, n):
    L = 256
    A = inputs.gaussian(m, n, 2027)
    t = oracle.make_tree(L, TREE4)
    QR_o, T_o = oracle.caqr(A, n, t, ld_pad=8)
    Ad = to_dev(A)
    del A
    qtree, info = ca.tsqr(Ad, ca.make_tree(L, TREE4))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    check(qr_err(Ad.cpu().numpy(), QR_o), 1e-12, (m, n))                      # R, every stored Y
    check(qtree_err(qtree.cpu().numpy(), T_o, QR_o, n, t, oracle.tree_counts), 1e-12, (m, n))   # every T


def test_calu_caqr_4096_benchmark_shape(ca):
    """CALU and CAQR of 4096 x 4096 (iid N(0,1)) with the benchmark's panel
    width, leaves and tree, against the full oracle (both oracle runs in two
    threads: the C code runs without the interpreter lock)."""
    import threading
    n, b, L = 4096, 128, bench.BENCH_LEAF_ROWS
    A = inputs.gaussian(n, n, 4096)
    t = oracle.make_tree(L, BENCH_TREE)
    out = {}
    th = [threading.Thread(target=lambda: out.__setitem__("lu", oracle.calu(A, b, t, ld_pad=8))),
          threading.Thread(target=lambda: out.__setitem__("qr", oracle.caqr(A, b, t, ld_pad=8)))]
    for x in th:
        x.start()
    tree = ca.make_tree(L, BENCH_TREE)
    Alu, Aqr = to_dev(A), to_dev(A)
    ipiv, info = ca.calu_factor(Alu, b, tree)
    qtree, qinfo = ca.caqr_factor(Aqr, b, tree)
    torch.cuda.synchronize()
    for x in th:
        x.join()
    LU_o, ipiv_o, info_o, nt = out["lu"]
    QR_o, T_o = out["qr"]
    assert nt == 0 and info_o == 0
    assert info.cpu().tolist() == [0, 0] and qinfo.cpu().tolist() == [0, 0]
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_o)            # all 32 panels' pivots
    check(lu_err(Alu.cpu().numpy(), LU_o), 1e-12, "CALU 4096")
    check(qr_err(Aqr.cpu().numpy(), QR_o, b), 1e-12, "CAQR 4096")
    check(qtree_err(qtree.cpu().numpy(), T_o, QR_o, b, t, oracle.tree_counts), 1e-12, "CAQR 4096 T")


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
    assert float(be.item()) <= 1e-14 and berr(A0, Xm, B0) < 1e-14
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
