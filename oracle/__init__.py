"""CPU oracle for tree-based LU (CALU) and QR (CAQR / TSQR) in FP64 (and the
same code built for FP32, used for the FP32 form of the batched path).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may load it.  The arithmetic lives in ``ca_oracle.c`` (plain C,
``-O2 -ffp-contract=off``); this module compiles it on first use and marshals
numpy arrays (column-major float64) through ``ctypes``.

Every function is pinned by tests against the mathematics (exact rational
GEPP, LAPACK QR and LU through numpy/scipy, uniqueness of R, identities of
the compact WY form); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ca_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libca_oracle.so")
_LIB32 = os.path.join(_HERE, "_build", "libca_oracle_f32.so")
_lock = threading.Lock()
_lib = None
_lib32 = None

MAXLEV = 8
BINARY = 0
FLAT = 1


class _Tree(ctypes.Structure):
    _fields_ = [
        ("leaf_rows", ctypes.c_int),
        ("nlevels", ctypes.c_int),
        ("fan_in", ctypes.c_int * MAXLEV),
        ("style", ctypes.c_int * MAXLEV),
        ("op_depth", ctypes.c_int),
        ("op_b", ctypes.c_int * 2),
        ("op_leaf_rows", ctypes.c_int * 2),
    ]


def build(force: bool = False) -> str:
    """Compile ``ca_oracle.c`` into ``oracle/_build/libca_oracle.so`` (FP64)
    and ``libca_oracle_f32.so`` (the same source with ORA_REAL=float)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    for lib, extra in ((_LIB, []), (_LIB32, ["-DORA_REAL=float"])):
        if (not force and os.path.exists(lib)
                and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
            continue
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared",
               "-fPIC", *extra, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return _LIB


def _load(dtype=np.float64):
    global _lib, _lib32
    with _lock:
        if np.dtype(dtype) == np.float32:
            if _lib32 is None:
                build()
                _lib32 = _declare(ctypes.CDLL(_LIB32))
            return _lib32
        if _lib is None:
            alt = os.environ.get("CA_ORACLE_LIB")  # a planted-mistake build (tests only)
            if alt:
                lib = ctypes.CDLL(alt)
            else:
                build()
                lib = ctypes.CDLL(_LIB)
            _lib = _declare(lib)
    return _lib


def _declare(lib):
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.ora_tree_counts.argtypes = [I, P, P, P]
    lib.ora_getf2.argtypes = [I, I, P, I, P, P]
    lib.ora_tslu_select.argtypes = [I, I, P, I, P, P, P]
    lib.ora_calu.argtypes = [I, I, P, I, I, P, P, P]
    lib.ora_getrs.argtypes = [I, I, P, I, P, P, I]
    lib.ora_geqrt.argtypes = [I, I, P, I, P, I]
    lib.ora_caqr_tcount.argtypes = [I, I, I, P]
    lib.ora_caqr_tcount.restype = ctypes.c_longlong
    lib.ora_caqr.argtypes = [I, I, P, I, I, P, P]
    lib.ora_geqrs.argtypes = [I, I, I, P, I, I, P, P, P, I]
    lib.ora_caqr_apply_qt.argtypes = [I, I, P, I, I, P, P, P, I, I]
    return lib


def make_tree(leaf_rows: int, levels=((0, BINARY),), op=()) -> dict:
    """A reduction tree: leaves of ``leaf_rows`` rows; ``levels`` is a list of
    (fan_in, style) from the bottom up; the last level merges all remaining
    nodes whatever its fan_in says.  ``op``: the reduction operator of the
    tournament's nodes, () for GEPP, or up to two (b, leaf_rows) pairs from
    the top down for the 2D multilevel CALU operator (each node factored by
    CALU with that block size over a binary tree of such leaves)."""
    return {"leaf_rows": int(leaf_rows), "levels": [(int(f), int(s)) for f, s in levels],
            "op": [(int(b), int(L)) for b, L in op]}


def _ctree(tree: dict) -> _Tree:
    t = _Tree()
    t.leaf_rows = tree["leaf_rows"]
    lv = tree["levels"]
    if not 1 <= len(lv) <= MAXLEV:
        raise ValueError("tree needs 1..8 levels")
    t.nlevels = len(lv)
    for i, (f, s) in enumerate(lv):
        t.fan_in[i] = f
        t.style[i] = s
    op = tree.get("op", [])
    if len(op) > 2:
        raise ValueError("operator depth 0..2")
    t.op_depth = len(op)
    for d, (b, L) in enumerate(op):
        t.op_b[d] = b
        t.op_leaf_rows[d] = L
    return t


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.array(a, dtype=np.float64, copy=True))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def tree_counts(m: int, tree: dict) -> tuple[int, int]:
    lib = _load()
    nl = ctypes.c_int()
    nm = ctypes.c_int()
    t = _ctree(tree)
    if lib.ora_tree_counts(m, ctypes.byref(t), ctypes.byref(nl), ctypes.byref(nm)):
        raise ValueError("bad tree")
    return nl.value, nm.value


def getf2(A):
    """Unblocked GEPP (LAPACK getf2).  Returns (LU, ipiv 1-based, info, nearties)."""
    lib = _load()
    A = _f64(A)
    m, n = A.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    nt = ctypes.c_long(0)
    info = lib.ora_getf2(m, n, _ptr(A), max(1, m), _ptr(ipiv), ctypes.byref(nt))
    return A, ipiv[: min(m, n)], info, nt.value


def tslu_select(P, tree: dict):
    """Tournament pivoting on an m x b panel.  Returns (rows chosen by the
    root in selection order, nearties)."""
    lib = _load()
    P = _f64(P)
    m, b = P.shape
    sel = np.zeros(max(1, min(m, b)), dtype=np.int32)
    nt = ctypes.c_long(0)
    t = _ctree(tree)
    k = lib.ora_tslu_select(m, b, _ptr(P), max(1, m), ctypes.byref(t), _ptr(sel), ctypes.byref(nt))
    if k < 0:
        raise ValueError(f"ora_tslu_select failed ({k})")
    return sel[:k], nt.value


def _arr(a, dtype) -> np.ndarray:
    return np.asfortranarray(np.array(a, dtype=dtype, copy=True))


def _padded(a, dtype, ld_pad: int):
    """A column-major copy of ``a`` whose leading dimension is m + ld_pad
    (marshalling only: the C code sees the same values through a larger lda;
    a leading dimension that is a large power of two makes the row-wise loops
    of the C code alias in the host cache).  Returns (buffer, view of the top
    m rows, lda)."""
    a = np.asarray(a)
    m, n = a.shape
    lda = max(1, m + int(ld_pad))
    buf = np.zeros((lda, n), dtype=dtype, order="F")
    buf[:m] = a
    return buf, buf[:m], lda


def calu(A, b: int, tree: dict, dtype=np.float64, ld_pad: int = 0):
    """CALU with tournament pivoting.  Returns (LU, ipiv 1-based, info, nearties).
    dtype float32: the FP32 build (every operation and pivot decision in FP32).
    ld_pad: rows of padding below the matrix in the buffer handed to the C
    code (same result; see ``_padded``)."""
    lib = _load(dtype)
    buf, A, lda = _padded(A, dtype, ld_pad)
    m, n = A.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    nt = ctypes.c_long(0)
    t = _ctree(tree)
    info = lib.ora_calu(m, n, _ptr(buf), lda, b, ctypes.byref(t), _ptr(ipiv), ctypes.byref(nt))
    if info < 0:
        raise ValueError(f"ora_calu failed ({info})")
    return np.asfortranarray(A), ipiv[: min(m, n)], info, nt.value


def getrs(LU, ipiv, B):
    lib = _load()
    LU = _f64(LU)
    B = _f64(B)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    n = LU.shape[0]
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.ora_getrs(n, B.shape[1], _ptr(LU), max(1, n), _ptr(ipiv), _ptr(B), max(1, n))
    return B


def geqrt(A):
    """Householder QR (geqr2) and T (larft).  Returns (QR, T)."""
    lib = _load()
    A = _f64(A)
    m, n = A.shape
    k = min(m, n)
    T = np.zeros((max(k, 1), max(k, 1)), order="F")
    lib.ora_geqrt(m, n, _ptr(A), max(1, m), _ptr(T), max(1, k))
    return A, T[:k, :k]


def caqr_tcount(m: int, n: int, b: int, tree: dict) -> int:
    lib = _load()
    t = _ctree(tree)
    c = lib.ora_caqr_tcount(m, n, b, ctypes.byref(t))
    if c < 0:
        raise ValueError("bad tree")
    return int(c)


def caqr(A, b: int, tree: dict, dtype=np.float64, ld_pad: int = 0):
    """CAQR (TSQR panels + tree update).  Returns (QR factors, T storage).
    dtype float32: the FP32 build.  ld_pad: as for ``calu``."""
    lib = _load(dtype)
    buf, A, lda = _padded(A, dtype, ld_pad)
    m, n = A.shape
    T = np.zeros(max(1, caqr_tcount(m, n, b, tree)), dtype=dtype)
    t = _ctree(tree)
    rc = lib.ora_caqr(m, n, _ptr(buf), lda, b, ctypes.byref(t), _ptr(T))
    if rc:
        raise ValueError(f"ora_caqr failed ({rc})")
    return np.asfortranarray(A), T


def tsqr(A, tree: dict):
    """TSQR = CAQR with one panel as wide as the matrix."""
    A = np.asarray(A)
    return caqr(A, A.shape[1], tree)


def geqrs(QR, T, b: int, tree: dict, B):
    """Least squares from CAQR factors; returns x (n x nrhs)."""
    lib = _load()
    QR = _f64(QR)
    B = _f64(B)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    m, n = QR.shape
    t = _ctree(tree)
    T = np.ascontiguousarray(T, dtype=np.float64)
    rc = lib.ora_geqrs(m, n, B.shape[1], _ptr(QR), max(1, m), b, ctypes.byref(t), _ptr(T), _ptr(B),
                       max(1, m))
    if rc:
        raise ValueError(f"ora_geqrs failed ({rc})")
    return B[:n]


def caqr_apply_qt(QR, T, b: int, tree: dict, C):
    """Q^T C for the CAQR factors (C is m x nc)."""
    lib = _load()
    QR = _f64(QR)
    C = _f64(C)
    if C.ndim == 1:
        C = C.reshape(-1, 1, order="F")
    m, n = QR.shape
    t = _ctree(tree)
    T = np.ascontiguousarray(T, dtype=np.float64)
    rc = lib.ora_caqr_apply_qt(m, n, _ptr(QR), max(1, m), b, ctypes.byref(t), _ptr(T), _ptr(C),
                               max(1, m), C.shape[1])
    if rc:
        raise ValueError(f"ora_caqr_apply_qt failed ({rc})")
    return C


# ---------------------------------------------------------------------------
# Helpers that unpack factors (plain definitions, used by the tests)
# ---------------------------------------------------------------------------

def lu_unpack(LU, ipiv):
    """(P, L, U) with P A = L U for LAPACK-layout factors."""
    LU = np.asarray(LU)
    m, n = LU.shape
    k = min(m, n)
    L = np.tril(LU[:, :k], -1) + np.eye(m, k)
    U = np.triu(LU[:k, :])
    perm = np.arange(m)
    for i, p in enumerate(np.asarray(ipiv)[:k]):
        p -= 1
        perm[i], perm[p] = perm[p], perm[i]
    return perm, L, U


def caqr_q(QR, T, b: int, tree: dict):
    """Explicit m x m Q of a CAQR factorization (Q = (Q^T)^T applied to I)."""
    m = QR.shape[0]
    QtI = caqr_apply_qt(QR, T, b, tree, np.eye(m))
    return QtI.T
