"""The element-wise comparison used by the GPU parity tests, checked on the
CPU: two correct computations of the same factorization (the oracle and a
LAPACK / BLAS computation of the same mathematics) agree far inside the
1e-12 bar, and a single wrong entry that a whole-matrix norm would let pass
(one element of the last, ragged panel; one Y element; one T element) is
caught."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1303_5837_gb300 import inputs
from tests import parity

TOL = 1e-12


def nopiv_lu(A, b):
    """Blocked LU without pivoting (BLAS products: another rounding order)."""
    A = A.copy()
    n = A.shape[1]
    for k in range(0, n, b):
        e = min(k + b, n)
        for j in range(k, e):
            A[j + 1:, j] /= A[j, j]
            A[j + 1:, j + 1:e] -= np.outer(A[j + 1:, j], A[j, j + 1:e])
        if e < n:
            L11 = np.tril(A[k:e, k:e], -1) + np.eye(e - k)
            A[k:e, e:] = np.linalg.solve(L11, A[k:e, e:])
            A[e:, e:] -= A[e:, k:e] @ A[k:e, e:]
    return A


@pytest.fixture(scope="module")
def lu_case():
    n, b = 700, 64                     # ragged last panel: 700 = 10 x 64 + 60
    A = inputs.gaussian(n, n, 5)
    tree = oracle.make_tree(128, [(2, 0), (0, 1)])
    LU, ipiv, info, nt = oracle.calu(A, b, tree)
    assert info == 0 and nt == 0
    perm, _, _ = oracle.lu_unpack(LU, ipiv)
    return A, LU, perm, b


def test_lu_err_two_correct_computations(lu_case):
    A, LU, perm, b = lu_case
    alt = nopiv_lu(A[perm], b)
    rep = parity.lu_err(alt, LU)
    assert rep["max"] < 1e-13, rep
    assert parity.lu_err(LU, LU)["max"] == 0.0


def test_lu_err_catches_one_wrong_entry(lu_case):
    _, LU, _, _ = lu_case
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    S = np.abs(L) @ np.abs(np.triu(LU))
    for (i, j) in [(699, 650), (690, 699), (3, 1)]:    # L and U of the ragged panel, an early L
        bad = LU.copy()
        scale = S[i, j] / abs(LU[j, j]) if i > j else S[i, j]
        bad[i, j] += 2e-11 * scale                     # 20 x the bar on its own scale
        if i > j:                                      # a whole-matrix norm check passes it
            assert np.linalg.norm(bad - LU) / np.linalg.norm(LU) < 1e-12
        rep = parity.lu_err(bad, LU)
        assert rep["max"] > TOL and rep["at"] == (i, j), rep


def test_lu_err_ledger_padding_and_pad_option(lu_case):
    A, LU, _, b = lu_case
    LU2, ipiv2, _, _ = oracle.calu(A, b, oracle.make_tree(128, [(2, 0), (0, 1)]), ld_pad=8)
    assert np.array_equal(LU2, LU)     # the padded leading dimension changes nothing


@pytest.fixture(scope="module")
def qr_case():
    m, n = 900, 600
    A = inputs.gaussian(m, n, 9)
    QR, T = oracle.caqr(A, 64, oracle.make_tree(m))      # one leaf: blocked Householder
    return A, QR, T


def test_qr_err_two_correct_computations(qr_case):
    A, QR, _ = qr_case
    (qr, tau), _ = sl.qr(A, mode="raw")                  # LAPACK geqrf, same convention
    rep = parity.qr_err(qr, QR, 64)
    assert rep["max"] < 1e-13, rep


def test_qr_err_catches_one_wrong_entry(qr_case):
    _, QR, _ = qr_case
    for (i, j) in [(899, 599), (10, 598), (599, 598)]:   # Y of the last column, R, Y
        bad = QR.copy()
        bad[i, j] += 1e-10 * max(1.0, abs(QR[i, j]))
        rep = parity.qr_err(bad, QR, 64)
        assert rep["max"] > TOL and rep["at"] == (i, j), rep


def test_qtree_err_catches_one_wrong_t_entry():
    m, n, b = 1000, 200, 48
    tree = oracle.make_tree(160, [(3, 1), (0, 0)])
    QR, T = oracle.caqr(inputs.gaussian(m, n, 10), b, tree)
    assert parity.qtree_err(T, T, QR, b, tree, oracle.tree_counts)["max"] == 0.0
    nz = np.flatnonzero(T)
    for k in (nz[-1], nz[len(nz) // 2]):
        bad = T.copy()
        bad[k] += 1e-9
        rep = parity.qtree_err(bad, T, QR, b, tree, oracle.tree_counts)
        assert rep["max"] > TOL, rep
    bad = T.copy()
    z = b * 3 + 7                                         # block 0, column 3, row 7: below the diagonal
    assert T[z] == 0.0
    bad[z] = 1e-300
    assert parity.qtree_err(bad, T, QR, b, tree, oracle.tree_counts)["max"] == np.inf


def test_solve_err():
    x = np.array([[1.0, 100.0], [2.0, -200.0]])
    y = x.copy()
    y[0, 1] += 1e-9
    rep = parity.solve_err(y, x)
    assert rep["at"] == (0, 1) and abs(rep["max"] - 5e-12) < 1e-15


def test_chunked_equals_whole(lu_case, qr_case, monkeypatch):
    A, LU, perm, b = lu_case
    alt = nopiv_lu(A[perm], b)
    Aq, QR, _ = qr_case
    (qr, _t), _ = sl.qr(Aq, mode="raw")
    whole = (parity.lu_err(alt, LU), parity.qr_err(qr, QR, 64))
    monkeypatch.setattr(parity, "CHUNK", 97)
    parts = (parity.lu_err(alt, LU), parity.qr_err(qr, QR, 64))
    for w, p in zip(whole, parts):
        assert w["max"] == p["max"] and w["at"] == p["at"]
        assert abs(w["frob"] - p["frob"]) <= 1e-12 * w["frob"]
