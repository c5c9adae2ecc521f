"""Element-wise comparison of factors (test helper; no factorization
arithmetic of its own beyond the scale of each element).

Every element of a result is compared with the oracle's, divided by the
size that first-order rounding analysis gives that element, so that one
wrong entry anywhere (a ragged last panel, one T block among hundreds) shows
up at its own scale instead of vanishing in a whole-matrix norm:

* LU (P A = L U): the computed factors of any backward-stable elimination
  with the same pivots satisfy L U = P A + E with |E| <= c n eps |L||U|
  (componentwise; LU backward error analysis).  An element U_ij is therefore
  compared on the scale (|L||U|)_ij, an element L_ij on (|L||U|)_ij / |U_jj|.
* QR (A = Q R, Householder, tree or not): column j of R carries an error of
  order eps ||A(:, j)||, and a reflector built from a sub-column x of the
  updated column j carries an error of order eps ||A(:, j)|| / ||x||.  R_ij is
  compared on ||R(:, j)|| (= ||A(:, j)||), every stored Y element of column j
  on ||R(:, j)|| / |R_jj| (|R_jj| is the norm of the sub-column the root's
  reflector was built from; the running maximum over the panel's earlier
  columns, whose reflectors were applied to it first), and column j of every
  T block on that scale times the block column's largest entry.

Each check returns the largest scaled difference with its location and the
Frobenius relative difference beside it; assertions print all three.
"""
from __future__ import annotations

import numpy as np


def _report(r: np.ndarray, d: np.ndarray, o: np.ndarray, label: str) -> dict:
    if r.size == 0:
        return {"what": label, "max": 0.0, "at": None, "frob": 0.0}
    i = np.unravel_index(int(np.argmax(r)), r.shape)
    no = float(np.linalg.norm(o))
    return {"what": label, "max": float(r[i]), "at": tuple(int(x) for x in i),
            "frob": float(np.linalg.norm(d)) / (no if no > 0 else 1.0)}


def _scaled(d: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """d / scale, where a zero scale demands an exact match (inf otherwise)."""
    out = np.zeros_like(d)
    pos = scale > 0
    out[pos] = d[pos] / scale[pos]
    out[~pos & (d != 0)] = np.inf
    return out


def _finite_pair(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    fg, fw = np.isfinite(got), np.isfinite(want)
    assert np.array_equal(fg, fw), "non-finite entries differ"
    return np.where(fw, got, 0.0), np.where(fw, want, 0.0), fw


CHUNK = 1 << 18   # rows per chunk for tall matrices


def _merge(reps, o_norm2: float, label: str) -> dict:
    best = max(reps, key=lambda r: r[0])
    d2 = sum(r[2] for r in reps)
    return {"what": label, "max": best[0], "at": best[1],
            "frob": float(np.sqrt(d2) / (np.sqrt(o_norm2) if o_norm2 > 0 else 1.0))}


def _chunk_rep(r: np.ndarray, d: np.ndarray, row0: int):
    if r.size == 0:
        return (0.0, None, 0.0)
    i = np.unravel_index(int(np.argmax(r)), r.shape)
    return (float(r[i]), (int(i[0]) + row0, int(i[1])), float(np.sum(d * d)))


def lu_err(got, want) -> dict:
    """Largest |got - want| over its componentwise scale for LAPACK-layout LU
    factors (unit L strictly below the diagonal, U on and above).  Where the
    oracle's factors hold non-finite values (an exactly zero pivot) those
    entries must coincide and the rest is compared column-relative."""
    got = np.asarray(got)
    want = np.asarray(want)
    m, n = want.shape
    k = min(m, n)
    fin_all = bool(np.isfinite(want).all())
    U = np.triu(np.asarray(want[:k, :], dtype=np.float64))
    aU = np.abs(U)
    udiag = np.abs(np.diag(U))
    colmax = np.abs(np.where(np.isfinite(want), want, 0.0)).max(axis=0, keepdims=True) if not fin_all else None
    reps, o2 = [], 0.0
    for r0 in range(0, max(m, 1), CHUNK):
        r1 = min(m, r0 + CHUNK)
        g, w, _ = _finite_pair(got[r0:r1], want[r0:r1])
        d = np.abs(g - w)
        o2 += float(np.sum(w * w))
        if not fin_all:
            scale = np.abs(w) + colmax
        else:
            rows = np.arange(r0, r1)[:, None]
            cols = np.arange(n)[None, :]
            lower = rows > cols
            Lc = np.where(rows[:, :k] > cols[:, :k], w[:, :k], 0.0)
            Lc[rows[:, 0] < k, rows[rows[:, 0] < k, 0]] = 1.0
            S = np.abs(Lc) @ aU                              # (|L||U|)_ij
            with np.errstate(divide="ignore", invalid="ignore"):
                scale = np.where(lower, S / np.concatenate([udiag, np.ones(n - k)])[None, :], S)
            scale[~np.isfinite(scale)] = 0.0
        reps.append(_chunk_rep(_scaled(d, scale), d, r0))
    label = "LU (componentwise, |L||U|)" if fin_all else "LU (column-relative, non-finite oracle)"
    return _merge(reps, o2, label)


def qr_col_scales(QR_o, n: int):
    """(||R(:, j)||, ||R(:, j)|| / |R_jj|) for the oracle's final R."""
    R = np.triu(np.asarray(QR_o, dtype=np.float64)[:n, :n])
    cn = np.linalg.norm(R, axis=0)
    rd = np.abs(np.diag(R))
    with np.errstate(divide="ignore", invalid="ignore"):
        ys = np.where(rd > 0, cn / rd, cn)
    return cn, ys


def _panel_cummax(ys, n: int, b: int):
    """Running maximum of the Y scales inside each panel of width b: a
    reflector of column j also carries the errors of the panel's earlier
    reflectors applied to its sub-column."""
    out = np.array(ys, dtype=np.float64, copy=True)
    for kb in range(0, n, b):
        out[kb: kb + b] = np.maximum.accumulate(out[kb: kb + b])
    return out


def qr_err(got, want, b: int | None = None) -> dict:
    """Largest scaled difference of a CAQR / TSQR factor array (R on and above
    the diagonal, every stored Y below it); b: the panel width (default: one
    panel)."""
    got = np.asarray(got)
    want = np.asarray(want)
    m, n = want.shape
    cn, ys = qr_col_scales(want, n)
    ys = _panel_cummax(ys, n, b or max(n, 1))
    reps, o2 = [], 0.0
    for r0 in range(0, max(m, 1), CHUNK):
        r1 = min(m, r0 + CHUNK)
        g, w, _ = _finite_pair(got[r0:r1], want[r0:r1])
        upper = np.arange(r0, r1)[:, None] <= np.arange(n)[None, :]
        scale = np.where(upper, cn[None, :], ys[None, :])
        d = np.abs(g - w)
        o2 += float(np.sum(w * w))
        reps.append(_chunk_rep(_scaled(d, scale), d, r0))
    return _merge(reps, o2, "QR (R: column norm, Y: column norm / |R_jj|)")


def _panel_blocks(m: int, n: int, b: int, tree: dict, tree_counts):
    """(first global column, width, number of b x b T blocks) per panel."""
    out = []
    for kb in range(0, n, b):
        nl, nm = tree_counts(m - kb, tree)
        out.append((kb, min(b, n - kb), nl + nm))
    return out


def qtree_err(T, T_o, QR_o, b: int, tree: dict, tree_counts) -> dict:
    """Largest scaled difference of the T blocks (layout of caqr_factor: per
    panel, nleaves + nmerges column-major b x b blocks).  Each T is upper
    triangular: the entries below a block's diagonal must be exactly zero."""
    T = np.asarray(T, dtype=np.float64).ravel()[: np.asarray(T_o).size]
    T_o = np.asarray(T_o, dtype=np.float64).ravel()
    assert T.size == T_o.size
    m, n = np.asarray(QR_o).shape
    _, ys = qr_col_scales(QR_o, n)
    ys = _panel_cummax(ys, n, b)
    scale = np.zeros_like(T_o)
    off = 0
    for kb, bk, nblk in _panel_blocks(m, n, b, tree, tree_counts):
        blk = T_o[off: off + nblk * b * b].reshape(nblk, b, b)     # [block, col, row]
        colmax = np.abs(blk).max(axis=2)                            # [block, col]
        s = np.zeros((nblk, b))
        s[:, :bk] = colmax[:, :bk] * ys[kb: kb + bk][None, :]
        sc = np.repeat(s[:, :, None], b, axis=2)                    # [block, col, row]
        sc[:, np.tril_indices(b, -1)[1], np.tril_indices(b, -1)[0]] = 0.0   # row > col: exact zeros
        scale[off: off + nblk * b * b] = sc.ravel()
        off += nblk * b * b
    assert off == T_o.size, (off, T_o.size)
    d = np.abs(T - T_o)
    return _report(_scaled(d, scale), d, T_o, "T blocks (column scale x block column max)")


def check(rep: dict, tol: float, ctx=None):
    assert rep["max"] <= tol, (ctx, rep)
    return rep


def solve_err(got, want) -> dict:
    """Largest |x - x_o| over the oracle solution's largest entry in the same
    column (the infinity-norm forward error of each right-hand side)."""
    g, w, _ = _finite_pair(got, want)
    d = np.abs(g - w)
    scale = np.broadcast_to(np.abs(w).max(axis=0, keepdims=True), w.shape)
    return _report(_scaled(d, scale), d, w, "solution (per right-hand side, inf-norm)")
