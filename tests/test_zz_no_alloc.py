"""tslu_noalloc: the TSLU entry point for callers that cannot allocate device
memory (their HBM is owned by another allocator, or cudaMalloc's implicit
device synchronization is not allowed on their path).  It must give the same
pivots and factors as tslu, which takes a caller-provided workspace, on two
calls in a row (the static scratch keeps the previous call's contents), and
reject a shape whose scratch would not fit before launching anything.

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1303_5837_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def to_dev(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_5837_gb300 import _binding
    L = _binding.load()
    L.tslu_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                               ctypes.POINTER(_binding.ca_tree_t), ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
    return L


def test_tslu_noalloc_matches_tslu_twice(lib):
    import paper_1303_5837_gb300 as ca
    m, n, L = 100_000, 64, 256
    tree = ca.make_tree(L, [(4, 0), (0, 0)])
    stream = torch.cuda.current_stream()
    for seed in (5, 6):  # two calls in a row, different inputs
        A = inputs.gaussian(m, n, seed)
        A_ref = to_dev(A)
        ipiv_ref, info_ref = ca.tslu(A_ref, tree)
        A_new = to_dev(A)
        ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
        info = torch.full((2,), -7, dtype=torch.int32, device="cuda")
        rc = lib.tslu_noalloc(m, n, ctypes.c_void_p(A_new.data_ptr()), A_new.stride(1),
                              ctypes.byref(tree), ctypes.c_void_p(ipiv.data_ptr()),
                              ctypes.c_void_p(info.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(ipiv, ipiv_ref)
        assert info.cpu().tolist() == info_ref.cpu().tolist() == [0, 0]
        d = torch.linalg.norm(A_new - A_ref) / torch.linalg.norm(A_ref)
        assert float(d) <= TOL


def test_tslu_noalloc_rejects_oversized(lib):
    import paper_1303_5837_gb300 as ca
    tree = ca.make_tree(128)
    A = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    # 50M rows in 128-row leaves need more than the static scratch
    rc = lib.tslu_noalloc(50_000_000, 128, ctypes.c_void_p(A.data_ptr()), 50_000_000,
                          ctypes.byref(tree), None, None, None)
    assert rc == -1001
