"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the factorizations: it only draws
matrices.  Every generator is deterministic in its seed (numpy PCG64) and
returns column-major (Fortran-order) float64 arrays, the layout of the C-ABI.

Workload families (the shapes and value distributions of the paper's
experiments and of the benchmark configurations):
  * ``gaussian``      iid N(0, 1) entries (square and tall-skinny panels);
  * ``conditioned``   A = U diag(s) V^T with U, V orthogonal (QR of a Gaussian
                      matrix with the sign of R's diagonal folded in) and
                      s_i = cond^(-i/(n-1)), so that cond_2(A) = cond;
  * ``int_matrix``    small-integer matrices for exact-rational brute force.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    """m x n iid N(0,1), column-major float64."""
    g = rng(seed)
    return np.asfortranarray(g.standard_normal((n, m)).T)


def int_matrix(m: int, n: int, seed: int, lo: int = -9, hi: int = 9) -> np.ndarray:
    g = rng(seed)
    return np.asfortranarray(g.integers(lo, hi + 1, size=(m, n)).astype(np.float64))


def _haar(n: int, g: np.random.Generator) -> np.ndarray:
    z = g.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * np.sign(np.diag(r))


def singular_values(n: int, cond: float) -> np.ndarray:
    if n == 1:
        return np.ones(1)
    return cond ** (-np.arange(n) / (n - 1))


def conditioned(n: int, cond: float, seed: int, device=None) -> np.ndarray:
    """A = U diag(s) V^T with cond_2(A) = cond.  With ``device`` (a torch CUDA
    device) the orthogonal factors are drawn and multiplied there in FP64
    (only to make large inputs quickly; the result is returned on the host)."""
    if device is None:
        g = rng(seed)
        U = _haar(n, g)
        V = _haar(n, g)
        s = singular_values(n, cond)
        return np.asfortranarray((U * s) @ V.T)
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = []
    for _ in range(2):
        z = torch.randn(n, n, dtype=torch.float64, device=device, generator=gen)
        q, r = torch.linalg.qr(z)
        out.append(q * torch.sign(torch.diagonal(r)))
    U, V = out
    s = torch.as_tensor(singular_values(n, cond), device=device)
    A = (U * s) @ V.T
    return np.asfortranarray(A.cpu().numpy())


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    return gaussian(n, nrhs, seed)
