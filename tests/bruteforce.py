"""Exact-rational brute force used to pin the oracle (no floating point).

Written from the definitions, independently of ``oracle/ca_oracle.c``:
GEPP with the first-maximum rule (LAPACK getf2), tournament pivoting over the
reduction tree (leaves of ``leaf_rows`` rows, levels of consecutive groups,
binary pairwise rounds or one flat merge, the last level taking everything),
and CALU panel by panel with exact elimination.
"""
from __future__ import annotations

from fractions import Fraction


def to_frac(A):
    return [[Fraction(int(v)) if float(v).is_integer() else Fraction(v) for v in row] for row in A]


def gepp(rows, ncols=None):
    """GEPP on a list of rows (Fractions).  Returns (labels in final order,
    factored rows, exact_tie_seen)."""
    W = [list(r) for r in rows]
    r = len(W)
    c = len(W[0]) if ncols is None else ncols
    lab = list(range(r))
    tie = False
    for j in range(min(r, c)):
        col = [abs(W[i][j]) for i in range(j, r)]
        mx = max(col)
        if mx != 0 and col.count(mx) > 1:
            tie = True
        p = j + col.index(mx)
        if W[p][j] == 0:
            continue
        W[j], W[p] = W[p], W[j]
        lab[j], lab[p] = lab[p], lab[j]
        for i in range(j + 1, r):
            l = W[i][j] / W[j][j]
            W[i][j] = l
            for q in range(j + 1, c):
                W[i][q] -= l * W[j][q]
    return lab, W, tie


def ipiv_from_order(order, k, n=None):
    """LAPACK 1-based swap sequence moving rows order[0..k) to the top of n rows."""
    n = len(order) if n is None else n
    pos = list(range(n))
    cur = list(range(n))
    ipiv = []
    for i in range(k):
        p = pos[order[i]]
        ipiv.append(p + 1)
        a, b = cur[i], cur[p]
        cur[i], cur[p] = b, a
        pos[b], pos[a] = i, p
    return ipiv


def _merge(panel, cands, b, op=()):
    """The node operator: GEPP (op empty), or exact CALU of the node's rows
    with block op[0][0], leaves of op[0][1] rows, a binary tree, and the
    operator op[1:] at its own nodes (the 2D multilevel CALU reduction)."""
    rows = [panel[i] for i in cands]
    k = min(len(rows), b)
    if not op:
        lab, _, tie = gepp(rows, b)
    else:
        (b1, L1), inner = op[0], op[1:]
        ipiv, _, tie = calu(rows, b1, L1, [(0, 0)], inner)
        lab = list(range(len(rows)))
        for i, p in enumerate(ipiv):
            lab[i], lab[p - 1] = lab[p - 1], lab[i]
    return [cands[l] for l in lab[:k]], tie


def tournament(panel, b, leaf_rows, levels, op=()):
    """Rows selected by tournament pivoting; ``levels`` = [(fan_in, style)]
    with style 0 = binary, 1 = flat; ``op`` the node operator (see _merge).
    Returns (selected rows, tie_seen)."""
    m = len(panel)
    tie = False
    nodes = []
    for r0 in range(0, m, leaf_rows):
        rows = list(range(r0, min(r0 + leaf_rows, m)))
        sel, t = _merge(panel, rows, b, op)
        tie |= t
        nodes.append(sel)
    for li, (f, style) in enumerate(levels):
        if li == len(levels) - 1:
            f = len(nodes)
        groups = [nodes[g:g + f] for g in range(0, len(nodes), f)]
        out = []
        for grp in groups:
            if style == 1:
                if len(grp) == 1:
                    out.append(grp[0])
                else:
                    sel, t = _merge(panel, [i for c in grp for i in c], b, op)
                    tie |= t
                    out.append(sel)
            else:
                cur = grp
                while len(cur) > 1:
                    nxt = []
                    for i in range(0, len(cur), 2):
                        if i + 1 < len(cur):
                            sel, t = _merge(panel, cur[i] + cur[i + 1], b, op)
                            tie |= t
                            nxt.append(sel)
                        else:
                            nxt.append(cur[i])
                    cur = nxt
                out.append(cur[0])
        nodes = out
    assert len(nodes) == 1
    return nodes[0], tie


def calu(A, b, leaf_rows, levels, op=()):
    """Exact CALU: returns (ipiv 1-based, LU rows in LAPACK layout, tie_seen)."""
    W = [list(r) for r in A]
    m = len(W)
    n = len(W[0])
    K = min(m, n)
    ipiv = []
    tie = False
    for kb in range(0, K, b):
        bk = min(b, K - kb)
        panel = [row[kb:kb + bk] for row in W[kb:]]
        sel, t = tournament(panel, bk, leaf_rows, levels, op)
        tie |= t
        piv = ipiv_from_order(sel, bk, m - kb)
        for i, p in enumerate(piv):
            p -= 1
            W[kb + i], W[kb + p] = W[kb + p], W[kb + i]
            ipiv.append(kb + p + 1)
        # exact elimination of the panel columns without further pivoting
        for j in range(kb, kb + bk):
            for i in range(j + 1, m):
                l = W[i][j] / W[j][j]
                W[i][j] = l
                for q in range(j + 1, n):
                    W[i][q] -= l * W[j][q]
    return ipiv, W, tie


def det(A):
    """Exact determinant (fraction-free elimination with row exchanges)."""
    W = [list(r) for r in A]
    n = len(W)
    d = Fraction(1)
    for j in range(n):
        p = next((i for i in range(j, n) if W[i][j] != 0), None)
        if p is None:
            return Fraction(0)
        if p != j:
            W[j], W[p] = W[p], W[j]
            d = -d
        d *= W[j][j]
        for i in range(j + 1, n):
            l = W[i][j] / W[j][j]
            for q in range(j, n):
                W[i][q] -= l * W[j][q]
    return d
