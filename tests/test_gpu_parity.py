"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle on the
same seeded inputs.

Pivots and other index results must match exactly; every element of the FP64
factors (L, U, R, every stored Y, every T) must match within 1e-12 of its own
first-order rounding scale (``tests/parity.py``: |L||U| componentwise for LU,
column norms for R and the reflectors), and every solution entry within 1e-12
of its right-hand side's largest entry.  The sizes span several leaves,
several tree levels, ragged last leaves and ragged last panels, and run in
seconds on the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1303_5837_gb300 import inputs
from tests.parity import check, lu_err, qr_err, qtree_err, solve_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


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


TREES = {
    "binary": [(0, 0)],
    "warp_cta_cluster_grid": [(2, 0), (4, 0), (0, 0)],
    "flat_top": [(4, 0), (0, 1)],
    "flat3_binary": [(3, 1), (0, 0)],
}


# ---------------------------------------------------------------------------
# TSLU
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,L", [(1024, 64, 128), (2000, 32, 256), (4133, 64, 256), (700, 16, 64),
                                   (333, 40, 333)])
@pytest.mark.parametrize("tname", sorted(TREES))
def test_tslu_pivots_and_factors(ca, m, n, L, tname):
    A = inputs.gaussian(m, n, m + n + L)
    lv = TREES[tname]
    LU_o, ipiv_o, info_o, nt = oracle.calu(A, n, oracle.make_tree(L, lv))
    assert nt == 0, "oracle saw a near tie on this seed"
    Ad = to_dev(A)
    ipiv, info = ca.tslu(Ad, ca.make_tree(L, lv))
    torch.cuda.synchronize()
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_o)
    assert info.cpu().tolist() == [info_o, 0]
    check(lu_err(to_host(Ad), LU_o), TOL)


# ---------------------------------------------------------------------------
# CALU
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,b,L,tname", [
    (1024, 1024, 64, 128, "binary"),            # the 1024^2, b=64, 128-row leaves case
    (1000, 1000, 64, 128, "warp_cta_cluster_grid"),
    (777, 500, 48, 96, "flat_top"),
    (400, 650, 32, 64, "flat3_binary"),
    (515, 515, 128, 256, "binary"),
])
def test_calu_parity(ca, m, n, b, L, tname):
    A = inputs.gaussian(m, n, 7 + m * n)
    lv = TREES[tname]
    LU_o, ipiv_o, info_o, nt = oracle.calu(A, b, oracle.make_tree(L, lv))
    assert nt == 0
    Ad = to_dev(A)
    ipiv, info = ca.calu_factor(Ad, b, ca.make_tree(L, lv))
    torch.cuda.synchronize()
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_o)
    assert info.cpu().tolist() == [info_o, 0]
    check(lu_err(to_host(Ad), LU_o), TOL)


# (m, n, b, leaf_rows, levels, operator): the 2D multilevel operator in the
# single-matrix path (one CTA per tournament node), matrices far larger than
# one CTA, several panels, ragged sizes
OP_SINGLE = [
    (1024, 1024, 64, 256, [(0, 0)], [(32, 64)]),
    (1500, 1200, 64, 256, [(4, 1), (0, 0)], [(32, 64), (8, 16)]),
    (3000, 200, 64, 128, [(0, 0)], [(16, 32)]),
    (2048, 2048, 64, 256, [(0, 0)], [(32, 64), (8, 16)]),
]


@pytest.mark.parametrize("m,n,b,L,lv,op", OP_SINGLE)
def test_calu_2d_operator_single_matrix(ca, m, n, b, L, lv, op):
    """calu_factor with the 2D multilevel reduction operator (Algorithm
    2D-ML-CALU, depth 1 and 2) against the oracle's node_factor: pivots
    exactly, every factor element within 1e-12 of its rounding scale; the
    operator changes the pivots of plain CALU on the same tree."""
    A = inputs.gaussian(m, n, 31 * m + n)
    LU_o, ipiv_o, info_o, nt = oracle.calu(A, b, oracle.make_tree(L, lv, op))
    assert nt == 0
    Ad = to_dev(A)
    ipiv, info = ca.calu_factor(Ad, b, ca.make_tree(L, lv, op))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [info_o, 0]
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_o)
    check(lu_err(to_host(Ad), LU_o), TOL, (m, n, b, op))
    _, ipiv_plain, _, _ = oracle.calu(A, b, oracle.make_tree(L, lv))
    assert not np.array_equal(ipiv_plain, ipiv_o)


def test_calu_zero_column_info(ca):
    A = inputs.gaussian(256, 256, 3)
    A[:, 70] = 0.0
    LU_o, ipiv_o, info_o, _ = oracle.calu(A, 32, oracle.make_tree(64))
    Ad = to_dev(A)
    ipiv, info = ca.calu_factor(Ad, 32, ca.make_tree(64))
    torch.cuda.synchronize()
    assert info_o == 71
    assert info.cpu().tolist()[0] == 71
    assert np.array_equal(ipiv.cpu().numpy()[:64], ipiv_o[:64])


def test_tslu_zero_column_single_cta_nodes(ca):
    """A column that is exactly zero in every node, on a panel whose 128
    leaves are each held by one CTA: no interchange and no update at that
    column, the same selections as the oracle, info at the first zero pivot."""
    A = inputs.gaussian(8192, 32, 5)
    A[:, 5] = 0.0
    tree = [(2, 0), (0, 0)]
    _, ipiv_o, info_o, nt = oracle.calu(A, 32, oracle.make_tree(64, tree))
    assert nt == 0 and info_o == 6
    ipiv, info = ca.tslu(to_dev(A), ca.make_tree(64, tree))
    torch.cuda.synchronize()
    assert info.cpu().tolist()[0] == 6
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_o)


def test_calu_nonfinite_status(ca):
    A = inputs.gaussian(128, 128, 4)
    A[5, 3] = np.nan
    Ad = to_dev(A)
    _, info = ca.calu_factor(Ad, 32, ca.make_tree(64))
    torch.cuda.synchronize()
    assert info.cpu().tolist()[1] & 1


def test_calu_padding_untouched(ca):
    m, n, lda = 300, 200, 320
    A = inputs.gaussian(m, n, 11)
    buf = torch.full((n, lda), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    Ad = buf.t()[:m]
    assert Ad.stride() == (1, lda)
    ca.calu_factor(Ad, 32, ca.make_tree(64))
    torch.cuda.synchronize()
    assert torch.isnan(buf[:, m:]).all()
    LU_o, _, _, _ = oracle.calu(A, 32, oracle.make_tree(64))
    check(lu_err(to_host(Ad), LU_o), TOL)


def test_calu_empty(ca):
    Ad = torch.empty((0, 5), dtype=torch.float64, device="cuda")
    ipiv, info = ca.calu_factor(Ad, 4, ca.make_tree(8))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]


def test_getrs(ca):
    n = 600
    A = inputs.gaussian(n, n, 21)
    B = inputs.rhs(n, 3, 22)
    tree = [(2, 0), (0, 0)]
    LU_o, ipiv_o, _, _ = oracle.calu(A, 64, oracle.make_tree(128, tree))
    x_o = oracle.getrs(LU_o, ipiv_o, B)
    Ad = to_dev(A)
    ipiv, _ = ca.calu_factor(Ad, 64, ca.make_tree(128, tree))
    Bd = to_dev(B)
    ca.calu_getrs(Ad, ipiv, Bd)
    torch.cuda.synchronize()
    check(solve_err(to_host(Bd), x_o), TOL)


# ---------------------------------------------------------------------------
# TSQR / CAQR
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,L", [(2048, 64, 256), (3001, 32, 256), (1000, 16, 64), (256, 64, 256),
                                   (4100, 128, 256),
                                   # last leaves of 20 and 12 rows: merges of R factors of unequal height
                                   (2068, 64, 256), (2060, 64, 128)])
@pytest.mark.parametrize("tname", sorted(TREES))
def test_tsqr_parity(ca, m, n, L, tname):
    A = inputs.gaussian(m, n, 5 * m + n)
    lv = TREES[tname]
    QR_o, T_o = oracle.tsqr(A, oracle.make_tree(L, lv))
    Ad = to_dev(A)
    qtree, info = ca.tsqr(Ad, ca.make_tree(L, lv))
    torch.cuda.synchronize()
    QR = to_host(Ad)
    t = oracle.make_tree(L, lv)
    check(qr_err(QR, QR_o), TOL)                                           # R and every stored Y
    check(qtree_err(qtree.cpu().numpy(), T_o, QR_o, n, t, oracle.tree_counts), TOL)   # every T block
    assert info.cpu().tolist() == [0, 0]


@pytest.mark.parametrize("m,n,b,L,tname", [
    (1024, 1024, 64, 128, "binary"),
    (1200, 700, 64, 128, "warp_cta_cluster_grid"),
    (900, 333, 32, 100, "flat_top"),
    (640, 256, 128, 256, "binary"),
])
def test_caqr_parity(ca, m, n, b, L, tname):
    A = inputs.gaussian(m, n, 13 + m + n)
    lv = TREES[tname]
    QR_o, T_o = oracle.caqr(A, b, oracle.make_tree(L, lv))
    Ad = to_dev(A)
    qtree, info = ca.caqr_factor(Ad, b, ca.make_tree(L, lv))
    torch.cuda.synchronize()
    check(qr_err(to_host(Ad), QR_o, b), TOL)
    check(qtree_err(qtree.cpu().numpy(), T_o, QR_o, b, oracle.make_tree(L, lv), oracle.tree_counts), TOL)
    assert info.cpu().tolist() == [0, 0]


def test_geqrs(ca):
    m, n, b, L = 1500, 400, 64, 128
    tree = [(2, 0), (0, 0)]
    A = inputs.gaussian(m, n, 31)
    B = inputs.rhs(m, 4, 32)
    QR_o, T_o = oracle.caqr(A, b, oracle.make_tree(L, tree))
    x_o = oracle.geqrs(QR_o, T_o, b, oracle.make_tree(L, tree), B)
    Ad = to_dev(A)
    t = ca.make_tree(L, tree)
    qtree, _ = ca.caqr_factor(Ad, b, t)
    Bd = to_dev(B)
    ca.caqr_geqrs(Ad, b, t, qtree, Bd)
    torch.cuda.synchronize()
    check(solve_err(to_host(Bd)[:n], x_o), TOL)


@pytest.mark.parametrize("nrhs", [1, 2, 3, 5, 8, 9, 40])
@pytest.mark.parametrize("tname", ["binary", "flat3_binary"])
def test_geqrs_nrhs(ca, nrhs, tname):
    """Q^T B through the tree with 1 to 40 right-hand sides (column groups of
    1, 2, 4 and 8, a ragged last group), ragged leaves (1337 = 8 x 160 + 57),
    a panel width that is not a multiple of 32 and a ragged last panel
    (300 = 6 x 48 + 12), binary merges and flat merges of three children."""
    m, n, b, L = 1337, 300, 48, 160
    tree = TREES[tname]
    A = inputs.gaussian(m, n, 41 + nrhs)
    B = inputs.rhs(m, nrhs, 42 + nrhs)
    QR_o, T_o = oracle.caqr(A, b, oracle.make_tree(L, tree))
    x_o = oracle.geqrs(QR_o, T_o, b, oracle.make_tree(L, tree), B)
    Ad = to_dev(A)
    t = ca.make_tree(L, tree)
    qtree, _ = ca.caqr_factor(Ad, b, t)
    Bd = to_dev(B)
    ca.caqr_geqrs(Ad, b, t, qtree, Bd)
    torch.cuda.synchronize()
    check(qr_err(to_host(Ad), QR_o, b), TOL)
    check(qtree_err(qtree.cpu().numpy(), T_o, QR_o, b, oracle.make_tree(L, tree), oracle.tree_counts), TOL)
    check(solve_err(to_host(Bd)[:n], x_o), TOL)


def test_repeat_is_deterministic(ca):
    A = inputs.gaussian(2048, 2048 // 4, 77)
    outs = []
    for _ in range(2):
        Ad = to_dev(A)
        ipiv, _ = ca.calu_factor(Ad, 64, ca.make_tree(256, [(2, 0), (0, 0)]))
        torch.cuda.synchronize()
        outs.append((to_host(Ad), ipiv.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
