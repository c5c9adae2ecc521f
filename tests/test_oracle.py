"""Pins of the CPU oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: exact
rational arithmetic (tests/bruteforce.py), LAPACK through numpy / scipy,
uniqueness of the QR factor R, the compact WY identity, closed-form tree
counts and the printed worked example under tests/golden/.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1303_5837_gb300 import inputs
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BIN, FLAT = oracle.BINARY, oracle.FLAT


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def tie_free_int(m, n, seed0, chk, span=9):
    """First seeded integer matrix whose exact computation sees no tie."""
    for s in range(seed0, seed0 + 500):
        A = inputs.int_matrix(m, n, s, -span, span)
        if not chk(A):
            return A
    raise RuntimeError("no tie-free matrix found")


# ----------------------------------------------------------------------------
# reduction-tree shape
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("m,L,levels,nl,nm", [
    (1024, 128, [(0, BIN)], 8, 7),                  # binary: nl - 1 merges
    (1000, 128, [(0, BIN)], 8, 7),                  # ragged last leaf
    (1024, 128, [(0, FLAT)], 8, 1),                 # one flat merge
    (1024, 128, [(4, FLAT), (0, FLAT)], 8, 3),      # 2 flat groups + root
    (1280, 128, [(4, FLAT), (0, BIN)], 10, 3 + 2),  # groups 4,4,2 then binary over 3
    (1024, 128, [(2, BIN), (2, BIN), (0, BIN)], 8, 7),
    (100, 128, [(0, BIN)], 1, 0),                   # a single leaf
])
def test_tree_counts(m, L, levels, nl, nm):
    assert oracle.tree_counts(m, oracle.make_tree(L, levels)) == (nl, nm)


# ----------------------------------------------------------------------------
# GEPP (leaf and merge operator)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("m,n", [(4, 4), (6, 4), (8, 8), (16, 8), (5, 9)])
def test_gepp_exact_rational(m, n):
    A = tie_free_int(m, n, 10 * m + n, lambda A: bf.gepp(bf.to_frac(A))[2])
    lab, W, _ = bf.gepp(bf.to_frac(A))
    LU, ipiv, info, _ = oracle.getf2(A)
    k = min(m, n)
    assert list(ipiv) == bf.ipiv_from_order(lab, k)
    exact = np.array([[float(v) for v in row] for row in W])
    assert np.allclose(LU, exact, rtol=1e-13, atol=1e-13)
    assert info == 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gepp_ties_take_first_maximum(seed):
    """Exact ties: the pivot is the first maximum in the current row order
    (LAPACK idamax); integers in [-2, 2] tie often, and every elimination
    step stays exact in FP64 for these small sizes."""
    A = inputs.int_matrix(6, 6, seed, -2, 2)
    lab, W, tie = bf.gepp(bf.to_frac(A))
    assert tie
    _, ipiv, _, _ = oracle.getf2(A)
    assert list(ipiv) == bf.ipiv_from_order(lab, 6)


def test_gepp_determinant():
    A = tie_free_int(8, 8, 7, lambda A: bf.gepp(bf.to_frac(A))[2])
    LU, ipiv, _, _ = oracle.getf2(A)
    sign = (-1) ** int(np.sum(ipiv != np.arange(1, 9)))
    d = sign * np.prod(np.diag(LU))
    assert abs(d - float(bf.det(bf.to_frac(A)))) <= 1e-10 * abs(d)


def test_gepp_matches_lapack():
    A = inputs.gaussian(96, 64, 3)
    LU, ipiv, info, nt = oracle.getf2(A)
    lu, piv = sla.lu_factor(A)
    assert nt == 0 and info == 0
    assert np.array_equal(ipiv, piv[:64] + 1)
    assert rel(LU, lu) < 1e-12


def test_gepp_zero_column_info():
    A = inputs.gaussian(6, 5, 1)
    A[:, 2] = 0.0
    A[:, 4] = A[:, 3]
    _, ipiv, info, _ = oracle.getf2(A)
    assert info == 3
    assert ipiv[2] == 3  # no swap at a zero column


# ----------------------------------------------------------------------------
# TSLU tournament pivoting
# ----------------------------------------------------------------------------

def test_tslu_one_leaf_is_gepp():
    P = inputs.gaussian(512, 32, 5)
    sel, nt = oracle.tslu_select(P, oracle.make_tree(512))
    _, ipiv, _, _ = oracle.getf2(P)
    order = np.arange(512)
    for i, p in enumerate(ipiv):
        order[[i, p - 1]] = order[[p - 1, i]]
    assert nt == 0
    assert np.array_equal(sel, order[:32])


TREES = [
    (4, [(0, BIN)]),
    (4, [(2, BIN), (0, BIN)]),
    (6, [(0, FLAT)]),
    (4, [(3, FLAT), (0, BIN)]),
    (5, [(3, BIN), (0, FLAT)]),
    (4, [(2, BIN), (2, FLAT), (0, BIN)]),
]


@pytest.mark.parametrize("L,levels", TREES)
@pytest.mark.parametrize("m", [32, 37])
def test_tslu_exact_rational(L, levels, m):
    b = 4
    A = tie_free_int(m, b, 100 + m + L, lambda A: bf.tournament(bf.to_frac(A), b, L, levels)[1],
                     span=999)
    want, _ = bf.tournament(bf.to_frac(A), b, L, levels)
    got, _ = oracle.tslu_select(A, oracle.make_tree(L, levels))
    assert list(got) == want


def test_tslu_selection_is_from_leaves():
    P = inputs.gaussian(2000, 16, 9)
    tree = oracle.make_tree(64, [(4, BIN), (0, BIN)])
    sel, _ = oracle.tslu_select(P, tree)
    assert len(set(sel.tolist())) == 16
    leaf_cands = set()
    for r0 in range(0, 2000, 64):
        s, _ = oracle.tslu_select(P[r0:r0 + 64], oracle.make_tree(64))
        leaf_cands |= set((s + r0).tolist())
    assert set(sel.tolist()) <= leaf_cands


def test_tslu_binary_levels_equal_global_binary():
    """With binary style and power-of-two fan-ins, levels only say where the
    merges run: the pivots equal those of one binary tree over the leaves."""
    P = inputs.gaussian(4096, 32, 11)
    a, _ = oracle.tslu_select(P, oracle.make_tree(64, [(0, BIN)]))
    b_, _ = oracle.tslu_select(P, oracle.make_tree(64, [(4, BIN), (2, BIN), (0, BIN)]))
    assert np.array_equal(a, b_)


# ----------------------------------------------------------------------------
# CALU
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,b,L,levels", [
    (12, 12, 4, 4, [(0, BIN)]),
    (14, 10, 3, 4, [(2, BIN), (0, FLAT)]),
    (10, 13, 4, 5, [(0, FLAT)]),
])
def test_calu_exact_rational(m, n, b, L, levels):
    A = tie_free_int(m, n, 300 + m * n, lambda A: bf.calu(bf.to_frac(A), b, L, levels)[2], span=99)
    ipiv_x, W, _ = bf.calu(bf.to_frac(A), b, L, levels)
    LU, ipiv, info, _ = oracle.calu(A, b, oracle.make_tree(L, levels))
    assert list(ipiv) == ipiv_x and info == 0
    exact = np.array([[float(v) for v in row] for row in W])
    assert np.allclose(LU, exact, rtol=1e-12, atol=1e-12)


def test_calu_one_leaf_is_gepp():
    A = inputs.gaussian(300, 300, 4)
    LU, ipiv, info, nt = oracle.calu(A, 32, oracle.make_tree(512))
    lu, piv = sla.lu_factor(A)
    assert nt == 0 and info == 0
    assert np.array_equal(ipiv, piv + 1)
    assert rel(LU, lu) < 1e-11


@pytest.mark.parametrize("m,n,b,L", [(256, 256, 32, 64), (300, 200, 32, 48), (150, 260, 16, 40)])
def test_calu_backward_error(m, n, b, L):
    A = inputs.gaussian(m, n, m + n)
    LU, ipiv, info, _ = oracle.calu(A, b, oracle.make_tree(L, [(2, BIN), (0, BIN)]))
    perm, Lf, U = oracle.lu_unpack(LU, ipiv)
    assert info == 0
    assert np.linalg.norm(A[perm] - Lf @ U) / np.linalg.norm(A) < 1e-14
    # growth stays moderate (tournament pivoting, paper Sec. 5.1)
    assert np.abs(U).max() / np.abs(A).max() < 50


def test_calu_getrs_solves():
    n = 200
    A = inputs.gaussian(n, n, 21)
    x_true = inputs.rhs(n, 3, 22)
    B = A @ x_true
    LU, ipiv, _, _ = oracle.calu(A, 32, oracle.make_tree(64))
    x = oracle.getrs(LU, ipiv, B)
    assert rel(x, np.linalg.solve(A, B)) < 1e-11
    r = B - A @ x
    bwd = np.abs(r).max() / (np.abs(A).sum(1).max() * np.abs(x).max() + np.abs(B).max())
    assert bwd < 1e-15


def test_calu_singular_info():
    A = inputs.gaussian(64, 64, 2)
    A[:, 10] = 0.0
    _, _, info, _ = oracle.calu(A, 16, oracle.make_tree(16))
    assert info == 11


# ----------------------------------------------------------------------------
# Householder QR, compact WY
# ----------------------------------------------------------------------------

def reflector_product(V, tau):
    m, k = V.shape
    Q = np.eye(m)
    for j in range(k):
        v = np.zeros(m)
        v[j] = 1.0
        v[j + 1:] = V[j + 1:, j]
        Q = Q @ (np.eye(m) - tau[j] * np.outer(v, v))
    return Q


@pytest.mark.parametrize("m,n", [(40, 12), (12, 12), (9, 14)])
def test_geqrt_matches_lapack_and_wy(m, n):
    A = inputs.gaussian(m, n, m * n)
    QR, T = oracle.geqrt(A)
    k = min(m, n)
    R = np.triu(QR[:k])
    R_lapack = np.linalg.qr(A, mode="r")
    assert rel(R, R_lapack[:k]) < 1e-13  # same larfg sign convention
    V = np.tril(QR[:, :k], -1)
    Y = V + np.eye(m, k)
    Q_wy = np.eye(m) - Y @ T @ Y.T
    Q_h = reflector_product(V, np.diag(T))
    assert rel(Q_wy, Q_h) < 1e-13
    assert np.allclose(np.triu(T), T)
    assert rel(Q_wy[:, :k] @ R, A) < 1e-14
    assert np.linalg.norm(Q_wy.T @ Q_wy - np.eye(m)) < 1e-13


def test_geqrt_zero_subcolumn_tau_zero():
    A = np.asfortranarray(np.triu(inputs.gaussian(6, 6, 8)))
    QR, T = oracle.geqrt(A)
    assert np.all(np.diag(T) == 0.0)
    assert np.array_equal(QR, A)


# ----------------------------------------------------------------------------
# TSQR / CAQR
# ----------------------------------------------------------------------------

def normalized_r(R):
    d = np.sign(np.diag(R))
    d[d == 0] = 1
    return d[:, None] * R


@pytest.mark.parametrize("m,n,L,levels", [
    (1000, 16, 64, [(0, BIN)]),
    (1000, 16, 64, [(4, BIN), (2, BIN), (0, BIN)]),
    (777, 8, 40, [(3, FLAT), (0, BIN)]),
    (513, 32, 32, [(0, FLAT)]),
])
def test_tsqr_r_unique(m, n, L, levels):
    A = inputs.gaussian(m, n, m + n)
    tree = oracle.make_tree(L, levels)
    QR, T = oracle.tsqr(A, tree)
    R = np.triu(QR[:n])
    Rl = np.linalg.qr(A, mode="r")
    assert rel(normalized_r(R), normalized_r(Rl)) < 1e-13
    # R^T R = A^T A
    assert rel(R.T @ R, A.T @ A) < 1e-13
    Q = oracle.caqr_q(QR, T, n, tree)
    assert rel(Q[:, :n] @ R, A) < 1e-14
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) < 1e-12


@pytest.mark.parametrize("m,n,b,L,levels", [
    (256, 256, 32, 64, [(0, BIN)]),
    (300, 200, 32, 48, [(2, BIN), (0, FLAT)]),
    (257, 129, 16, 33, [(0, BIN)]),
])
def test_caqr_factorization(m, n, b, L, levels):
    A = inputs.gaussian(m, n, 7 * m + n)
    tree = oracle.make_tree(L, levels)
    QR, T = oracle.caqr(A, b, tree)
    R = np.triu(QR[:n])
    assert rel(normalized_r(R), normalized_r(np.linalg.qr(A, mode="r"))) < 1e-12
    Q = oracle.caqr_q(QR, T, b, tree)
    assert rel(Q[:, :n] @ R, A) < 1e-14
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) < 1e-12


def test_caqr_one_leaf_is_householder():
    """One leaf per panel: CAQR is blocked Householder QR, whose R equals
    LAPACK's without any sign normalisation."""
    A = inputs.gaussian(200, 120, 12)
    QR, _ = oracle.caqr(A, 32, oracle.make_tree(256))
    assert rel(np.triu(QR[:120]), np.linalg.qr(A, mode="r")) < 1e-13


def test_caqr_tree_storage_layout():
    """Merge Y blocks overwrite the non-first children's R rows; the final R
    sits in the panel's top rows, and T blocks follow the tree counts."""
    m, n, b, L = 256, 32, 32, 64
    tree = oracle.make_tree(L)
    A = inputs.gaussian(m, n, 1)
    QR, T = oracle.tsqr(A, tree)
    nl, nm = oracle.tree_counts(m, tree)
    assert T.size == (nl + nm) * b * b
    Tb = T.reshape(nl + nm, b, b).transpose(0, 2, 1)  # column-major blocks
    for blk in Tb:
        assert np.allclose(np.tril(blk, -1), 0)
        assert np.all((np.diag(blk) >= 0) & (np.diag(blk) <= 2))  # tau in [0, 2]


def test_geqrs_least_squares():
    m, n = 400, 120
    A = inputs.gaussian(m, n, 30)
    B = inputs.rhs(m, 2, 31)
    tree = oracle.make_tree(64, [(2, BIN), (0, BIN)])
    QR, T = oracle.caqr(A, 32, tree)
    x = oracle.geqrs(QR, T, 32, tree, B)
    x_ref = np.linalg.lstsq(A, B, rcond=None)[0]
    assert rel(x, x_ref) < 1e-12
    r = B - A @ x
    assert np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r)) < 1e-14


# ----------------------------------------------------------------------------
# golden worked example
# ----------------------------------------------------------------------------

def test_golden_tournament_example():
    """Hand-worked tournament (tests/golden/tslu_8x2.json): every node's GEPP
    done by hand in the file's comments."""
    with open(os.path.join(GOLDEN, "tslu_8x2.json")) as f:
        g = json.load(f)
    A = np.array(g["A"], dtype=np.float64)
    tree = oracle.make_tree(g["leaf_rows"], [tuple(x) for x in g["levels"]])
    sel, _ = oracle.tslu_select(A, tree)
    assert sel.tolist() == g["selected"]


# ---------------------------------------------------------------------------
# the FP32 build of the oracle (same source, ORA_REAL=float): pinned to the
# FP64 build, which is pinned above.  Where FP32 takes no near-tie decision,
# its pivots must be the FP64 pivots and its factors the FP64 factors to FP32
# accuracy; R of a QR is unique, so it must agree to FP32 accuracy anyway.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,b,L,levels", [(96, 96, 16, 32, [(0, 0)]), (300, 40, 40, 64, [(2, 1), (0, 0)]),
                                            (200, 200, 32, 64, [(0, 1)])])
def test_fp32_oracle_agrees_with_fp64(m, n, b, L, levels):
    tree = oracle.make_tree(L, levels)
    checked = 0
    for seed in range(6):
        A = inputs.gaussian(m, n, 4000 + seed)
        LU64, ip64, _, _ = oracle.calu(A, b, tree)
        LU32, ip32, _, nt32 = oracle.calu(A, b, tree, dtype=np.float32)
        assert LU32.dtype == np.float32
        if nt32 == 0:
            checked += 1
            assert np.array_equal(ip32, ip64)
            assert np.linalg.norm(LU32 - LU64) / np.linalg.norm(LU64) < 2e-5
        QR64, T64 = oracle.caqr(A, b, tree)
        QR32, T32 = oracle.caqr(A, b, tree, dtype=np.float32)
        k = min(m, n)
        R64, R32 = np.triu(QR64[:k]), np.triu(QR32[:k])
        assert np.linalg.norm(R32 - R64) / np.linalg.norm(R64) < 2e-5
        assert np.linalg.norm(T32 - T64) / np.linalg.norm(T64) < 2e-5
    assert checked >= 2


def test_fp32_oracle_is_single_precision():
    """Sums below FP32 resolution vanish in the FP32 build and not in FP64
    (the build really computes in float): GEPP of [[1, 1], [1, 1 + 2^-30]]."""
    A = np.array([[1.0, 1.0], [1.0, 1.0 + 2.0 ** -30]])
    LU64, _, info64, _ = oracle.calu(A, 2, oracle.make_tree(2))
    LU32, _, info32, _ = oracle.calu(A, 2, oracle.make_tree(2), dtype=np.float32)
    assert LU64[1, 1] == 2.0 ** -30 and info64 == 0
    assert LU32[1, 1] == 0.0 and info32 == 2


# ---------------------------------------------------------------------------
# the 2D multilevel CALU reduction operator (every tournament node factored
# by CALU of the level below instead of GEPP)
# ---------------------------------------------------------------------------
OPS = [
    [(2, 4)],             # one level below: CALU with b = 2 over 4-row leaves
    [(3, 3)],
    [(4, 8), (2, 4)],     # two levels below
]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("m,n,b,L,levels", [(16, 12, 4, 8, [(0, BIN)]), (20, 9, 4, 8, [(0, FLAT)]),
                                            (18, 18, 6, 12, [(2, BIN), (0, BIN)])])
def test_calu_2d_operator_exact_rational(op, m, n, b, L, levels):
    A = tie_free_int(m, n, 500 + m * n + len(op),
                     lambda A: bf.calu(bf.to_frac(A), b, L, levels, op)[2], span=99)
    ipiv_x, W, _ = bf.calu(bf.to_frac(A), b, L, levels, op)
    LU, ipiv, info, _ = oracle.calu(A, b, oracle.make_tree(L, levels, op))
    assert list(ipiv) == ipiv_x and info == 0
    exact = np.array([[float(v) for v in row] for row in W])
    assert np.allclose(LU, exact, rtol=1e-12, atol=1e-12)


def test_calu_2d_operator_degenerates_to_gepp():
    """An operator whose CALU has one panel and one leaf per node is GEPP."""
    A = inputs.gaussian(400, 96, 21)
    tree = oracle.make_tree(64, [(2, BIN), (0, BIN)])
    op_tree = oracle.make_tree(64, [(2, BIN), (0, BIN)], op=[(32, 1024)])
    LU, ipiv, _, nt = oracle.calu(A, 32, tree)
    LU2, ipiv2, _, nt2 = oracle.calu(A, 32, op_tree)
    assert nt == 0 and nt2 == 0
    assert np.array_equal(ipiv, ipiv2)
    assert np.array_equal(LU, LU2)


def test_calu_2d_operator_changes_pivots_and_stays_stable():
    """A genuine inner level picks other pivots than GEPP at the nodes; the
    factorization stays backward stable, with growth within the soft bands
    of the paper's experiments (Sec. 5.1: growth of the same order as GEPP)."""
    n, b, L = 256, 32, 64
    tree = oracle.make_tree(L, [(0, BIN)])
    op_tree = oracle.make_tree(L, [(0, BIN)], op=[(8, 16)])
    diff = 0
    for seed in range(3):
        A = inputs.gaussian(n, n, 60 + seed)
        LU, ipiv, _, _ = oracle.calu(A, b, tree)
        LU2, ipiv2, info2, _ = oracle.calu(A, b, op_tree)
        diff += int(not np.array_equal(ipiv, ipiv2))
        perm, Lf, U = oracle.lu_unpack(LU2, ipiv2)
        assert info2 == 0
        assert np.linalg.norm(A[perm] - Lf @ U) / np.linalg.norm(A) < 1e-13
        _, _, U0 = oracle.lu_unpack(*oracle.getf2(A)[:2])
        g_gepp = np.abs(U0).max() / np.abs(A).max()
        g_2d = np.abs(U).max() / np.abs(A).max()
        assert 0.002 < g_2d / g_gepp < 2.4 * 4
        assert np.abs(Lf).max() <= 64.0           # |L| stays bounded (tournament pivoting)
    assert diff >= 1


def test_caqr_rejects_reduction_operator():
    A = inputs.gaussian(64, 32, 1)
    with pytest.raises(ValueError):
        oracle.caqr(A, 16, oracle.make_tree(32, op=[(4, 8)]))
