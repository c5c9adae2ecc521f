"""Thin Python binding of the C-ABI in ``include/ca_gb300.h``.

Argument marshalling only: every computation runs in ``libcagb300.so``.
Matrices are torch CUDA float64 tensors in column-major layout (shape
(m, n), stride (1, lda)); ``colmajor`` makes such a tensor.  Work is
enqueued on the current torch CUDA stream.  If the library is missing the
calls raise; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

MAX_LEVELS = 8
BINARY = 0
FLAT = 1

CA_OK = 0
CA_ERR_WORKSPACE = -1001
CA_ERR_UNSUPPORTED = -1002
CA_ERR_LAUNCH = -1003
CA_ERR_TREE = -1004
CA_ERR_BATCH_ITEM = -1005
CA_STATUS_NONFINITE = 1
CA_STATUS_SOLVE_TIMEOUT = 16
CA_STATUS_REFACTORED = 32
CA_REFINE_CLASSIC = 0
CA_REFINE_GMRES = 1
CA_REFINE_AUTO = 2
REFINE = {"classic": CA_REFINE_CLASSIC, "gmres": CA_REFINE_GMRES, "auto": CA_REFINE_AUTO}
CA_BATCH_CALU = 0
CA_BATCH_CAQR = 1
CA_DTYPE_F64 = 0
CA_DTYPE_F32 = 1


class CaError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} returned {code}: {msg}")
        self.code = code


class ca_tree_t(ctypes.Structure):
    _fields_ = [
        ("leaf_rows", ctypes.c_int),
        ("nlevels", ctypes.c_int),
        ("fan_in", ctypes.c_int * MAX_LEVELS),
        ("style", ctypes.c_int * MAX_LEVELS),
        ("op_depth", ctypes.c_int),
        ("op_b", ctypes.c_int * 2),
        ("op_leaf_rows", ctypes.c_int * 2),
    ]


class ca_batch_item_t(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_int),
        ("m", ctypes.c_int),
        ("n", ctypes.c_int),
        ("lda", ctypes.c_int),
        ("A", ctypes.c_void_p),
        ("ipiv", ctypes.c_void_p),
        ("qtree", ctypes.c_void_p),
        ("info", ctypes.c_void_p),
        ("b", ctypes.c_int),
        ("tree", ca_tree_t),
    ]


def make_tree(leaf_rows: int, levels=((0, BINARY),), op=()) -> ca_tree_t:
    """Reduction tree: leaves of ``leaf_rows`` rows, then ``levels`` as
    (fan_in, style) pairs from the bottom up (the last level merges all).
    ``op``: the nodes' reduction operator, () for GEPP or up to two
    (b, leaf_rows) pairs for the 2D multilevel CALU operator (batched CALU)."""
    t = ca_tree_t()
    op = list(op)
    if len(op) > 2:
        raise ValueError("operator depth 0..2")
    t.op_depth = len(op)
    for d, (ob, oL) in enumerate(op):
        t.op_b[d] = int(ob)
        t.op_leaf_rows[d] = int(oL)
    t.leaf_rows = int(leaf_rows)
    levels = list(levels)
    if not 1 <= len(levels) <= MAX_LEVELS:
        raise ValueError("1..8 levels")
    t.nlevels = len(levels)
    for i, (f, s) in enumerate(levels):
        t.fan_in[i] = int(f)
        t.style[i] = int(s)
    return t


_lib = None

SYMBOLS = ("ca_strerror", "ca_calu_workspace", "ca_caqr_workspace", "ca_geqrs_workspace",
           "calu_factor", "tslu", "calu_getrs", "caqr_factor", "tsqr", "caqr_geqrs",
           "ca_prof_enable", "ca_prof_read", "ca_launch_count", "ca_kernel_class_name",
           "ca_gemm_mixed_workspace", "ca_gemm_minus_mixed", "ca_calu_mixed_workspace",
           "calu_factor_mixed", "ca_gesv_mixed_workspace", "calu_gesv_mixed", "ca_caqr_mixed_workspace",
           "caqr_factor_mixed", "ca_batched_plan", "ca_batched_factor", "ca_solve_status",
           "ca_getrs_workspace", "ca_test_solve_hook", "tslu_noalloc", "ca_peak_probe",
           "ca_gels_mixed_workspace", "caqr_gels_mixed")
KERNEL_CLASSES = ("tslu_node", "laswp", "lu_finish", "trsm_u12", "gemm_fp64", "tsqr_node",
                  "tree_apply", "solve", "split_bf16", "gemm_tc", "refine", "batched",
                  "tree_narrow")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcagb300.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    I, P, S = ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    PS = ctypes.POINTER(ctypes.c_size_t)
    T = ctypes.POINTER(ca_tree_t)
    L.ca_strerror.argtypes = [I]
    L.ca_strerror.restype = ctypes.c_char_p
    L.ca_calu_workspace.argtypes = [I, I, I, T, PS]
    L.ca_caqr_workspace.argtypes = [I, I, I, T, PS, PS]
    L.ca_geqrs_workspace.argtypes = [I, I, I, I, T, PS]
    L.calu_factor.argtypes = [I, I, P, I, I, T, P, P, S, P, P]
    L.tslu.argtypes = [I, I, P, I, T, P, P, S, P, P]
    L.calu_getrs.argtypes = [I, I, P, I, P, P, I, P, S, P]
    L.ca_getrs_workspace.argtypes = [I, I, PS]
    L.ca_test_solve_hook.argtypes = [ctypes.c_longlong, I]
    L.ca_test_solve_hook.restype = None
    L.ca_peak_probe.argtypes = [I, I, I, P, P]
    L.ca_gels_mixed_workspace.argtypes = [I, I, I, I, T, I, I, PS, PS]
    L.caqr_gels_mixed.argtypes = [I, I, I, P, I, I, T, I, I, P, I, P, S, P, I, P, I, P, S, I, ctypes.c_double,
                                  P, P, P, P]
    L.caqr_factor.argtypes = [I, I, P, I, I, T, P, S, P, S, P, P]
    L.tsqr.argtypes = [I, I, P, I, T, P, S, P, S, P, P]
    L.caqr_geqrs.argtypes = [I, I, I, P, I, I, T, P, S, P, I, P, S, P]
    L.ca_gemm_mixed_workspace.argtypes = [I, I, I, I, I, PS]
    L.ca_gemm_minus_mixed.argtypes = [I, I, I, P, I, P, I, P, I, I, I, P, S, P, P]
    L.ca_calu_mixed_workspace.argtypes = [I, I, I, T, I, I, PS]
    L.calu_factor_mixed.argtypes = [I, I, P, I, I, T, I, I, P, P, S, P, P]
    L.ca_gesv_mixed_workspace.argtypes = [I, I, I, T, I, I, I, PS]
    L.calu_gesv_mixed.argtypes = [I, I, P, I, I, T, I, I, I, P, I, P, P, I, P, I, P, S, I,
                                  ctypes.c_double, P, P, P, P]
    L.ca_caqr_mixed_workspace.argtypes = [I, I, I, T, I, I, PS, PS]
    L.caqr_factor_mixed.argtypes = [I, I, P, I, I, T, I, I, P, S, P, S, P, P]
    L.ca_batched_plan.argtypes = [I, ctypes.POINTER(ca_batch_item_t), I, P, PS, PS]
    L.ca_batched_factor.argtypes = [P, P, P, S, P]
    L.ca_solve_status.argtypes = [P, ctypes.POINTER(ctypes.c_int), P]
    L.ca_prof_enable.argtypes = [I, I]
    L.ca_prof_read.argtypes = [I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]
    L.ca_launch_count.argtypes = [I]
    L.ca_launch_count.restype = ctypes.c_longlong
    L.ca_kernel_class_name.argtypes = [I]
    L.ca_kernel_class_name.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(fn: str, rc: int):
    if rc != CA_OK:
        raise CaError(fn, rc, load().ca_strerror(rc).decode())


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Column-major copy of a 2-D tensor (shape kept, stride (1, m))."""
    return t.t().contiguous().t()


def _mat(A: torch.Tensor, name: str):
    if A.dim() != 2 or A.dtype != torch.float64 or not A.is_cuda:
        raise TypeError(f"{name} must be a 2-D CUDA float64 tensor")
    m, n = A.shape
    if m > 0 and n > 0 and A.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    lda = A.stride(1) if n > 1 else max(1, m)
    return m, n, max(lda, max(1, m))


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _buf(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(1, (nbytes + 7) // 8), dtype=torch.float64, device=device)


# ---------------------------------------------------------------------------
# workspace queries
# ---------------------------------------------------------------------------

def ca_calu_workspace(m: int, n: int, b: int, tree: ca_tree_t) -> int:
    out = ctypes.c_size_t(0)
    _check("ca_calu_workspace", load().ca_calu_workspace(m, n, b, ctypes.byref(tree), ctypes.byref(out)))
    return out.value


def ca_caqr_workspace(m: int, n: int, b: int, tree: ca_tree_t) -> tuple[int, int]:
    q = ctypes.c_size_t(0)
    w = ctypes.c_size_t(0)
    _check("ca_caqr_workspace",
           load().ca_caqr_workspace(m, n, b, ctypes.byref(tree), ctypes.byref(q), ctypes.byref(w)))
    return q.value, w.value


def ca_geqrs_workspace(m: int, n: int, nrhs: int, b: int, tree: ca_tree_t) -> int:
    w = ctypes.c_size_t(0)
    _check("ca_geqrs_workspace", load().ca_geqrs_workspace(m, n, nrhs, b, ctypes.byref(tree), ctypes.byref(w)))
    return w.value


# ---------------------------------------------------------------------------
# entry points (same names as the C-ABI)
# ---------------------------------------------------------------------------

def calu_factor(A: torch.Tensor, b: int, tree: ca_tree_t, ipiv=None, work=None, dev_info=None,
                stream=None):
    """CALU in place on A.  Returns (ipiv int32[min(m,n)], dev_info int32[2])."""
    m, n, lda = _mat(A, "A")
    dev = A.device
    if ipiv is None:
        ipiv = torch.empty(max(1, min(m, n)), dtype=torch.int32, device=dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    if work is None:
        work = _buf(ca_calu_workspace(m, n, b, tree), dev)
    rc = load().calu_factor(m, n, _ptr(A), lda, b, ctypes.byref(tree), _ptr(ipiv), _ptr(work),
                            work.numel() * work.element_size(), _ptr(dev_info), _stream(stream))
    _check("calu_factor", rc)
    return ipiv[: min(m, n)], dev_info


def tslu(A: torch.Tensor, tree: ca_tree_t, ipiv=None, work=None, dev_info=None, stream=None):
    m, n, lda = _mat(A, "A")
    dev = A.device
    if ipiv is None:
        ipiv = torch.empty(max(1, min(m, n)), dtype=torch.int32, device=dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    if work is None:
        work = _buf(ca_calu_workspace(m, n, max(n, 1), tree), dev)
    rc = load().tslu(m, n, _ptr(A), lda, ctypes.byref(tree), _ptr(ipiv), _ptr(work),
                     work.numel() * work.element_size(), _ptr(dev_info), _stream(stream))
    _check("tslu", rc)
    return ipiv[: min(m, n)], dev_info


def ca_getrs_workspace(n: int, nrhs: int) -> int:
    w = ctypes.c_size_t(0)
    _check("ca_getrs_workspace", load().ca_getrs_workspace(n, nrhs, ctypes.byref(w)))
    return w.value


def calu_getrs(LU: torch.Tensor, ipiv: torch.Tensor, B: torch.Tensor, work=None, stream=None):
    """Solve from CALU factors; B (n x nrhs) is overwritten with X.  work: the
    solve workspace (ca_getrs_workspace bytes; made here when None)."""
    n, _, lda = _mat(LU, "LU")
    nb, nrhs, ldb = _mat(B, "B")
    if work is None:
        work = _buf(ca_getrs_workspace(n, nrhs), LU.device)
    rc = load().calu_getrs(n, nrhs, _ptr(LU), lda, _ptr(ipiv), _ptr(B), ldb, _ptr(work),
                           work.numel() * work.element_size(), _stream(stream))
    _check("calu_getrs", rc)
    return B


def caqr_factor(A: torch.Tensor, b: int, tree: ca_tree_t, qtree=None, work=None, dev_info=None,
                stream=None):
    """CAQR in place on A.  Returns (qtree float64 tensor, dev_info)."""
    m, n, lda = _mat(A, "A")
    dev = A.device
    qb, wb = ca_caqr_workspace(m, n, b, tree)
    if qtree is None:
        qtree = _buf(qb, dev)
    if work is None:
        work = _buf(wb, dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    rc = load().caqr_factor(m, n, _ptr(A), lda, b, ctypes.byref(tree), _ptr(qtree),
                            qtree.numel() * 8, _ptr(work), work.numel() * work.element_size(),
                            _ptr(dev_info), _stream(stream))
    _check("caqr_factor", rc)
    return qtree, dev_info


def tsqr(A: torch.Tensor, tree: ca_tree_t, qtree=None, work=None, dev_info=None, stream=None):
    m, n, lda = _mat(A, "A")
    dev = A.device
    qb, wb = ca_caqr_workspace(m, n, max(n, 1), tree)
    if qtree is None:
        qtree = _buf(qb, dev)
    if work is None:
        work = _buf(wb, dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    rc = load().tsqr(m, n, _ptr(A), lda, ctypes.byref(tree), _ptr(qtree), qtree.numel() * 8,
                     _ptr(work), work.numel() * work.element_size(), _ptr(dev_info), _stream(stream))
    _check("tsqr", rc)
    return qtree, dev_info


def caqr_geqrs(QR: torch.Tensor, b: int, tree: ca_tree_t, qtree: torch.Tensor, B: torch.Tensor,
               work=None, stream=None):
    """Least squares from CAQR factors; B (m x nrhs) is overwritten, X = B[:n]."""
    m, n, lda = _mat(QR, "QR")
    mb, nrhs, ldb = _mat(B, "B")
    if work is None:
        work = _buf(ca_geqrs_workspace(m, n, nrhs, b, tree), QR.device)
    rc = load().caqr_geqrs(m, n, nrhs, _ptr(QR), lda, b, ctypes.byref(tree), _ptr(qtree),
                           qtree.numel() * 8, _ptr(B), ldb, _ptr(work),
                           work.numel() * work.element_size(), _stream(stream))
    _check("caqr_geqrs", rc)
    return B


def ca_solve_status(work: torch.Tensor, stream=None) -> bool:
    """Synchronizes the stream; True if the last solve that used this solve
    workspace (of calu_getrs or caqr_geqrs) gave up waiting for a block's
    ready flag (its right-hand sides are then only partly solved)."""
    t = ctypes.c_int(0)
    _check("ca_solve_status", load().ca_solve_status(_ptr(work), ctypes.byref(t), _stream(stream)))
    return bool(t.value)


def ca_peak_probe(dtype: int, blocks: int, iters: int, out: torch.Tensor, stream=None):
    """Enqueue the FMA peak probe (16 * iters * blocks * 256 flops)."""
    _check("ca_peak_probe", load().ca_peak_probe(int(dtype), int(blocks), int(iters), _ptr(out), _stream(stream)))


def ca_test_solve_hook(wait_cycles: int = 0, withhold: bool = False):
    """Test hook: withhold=True makes the next dependency-ordered solves leave
    their first block unpublished, so their waits run out after wait_cycles."""
    load().ca_test_solve_hook(int(wait_cycles), 1 if withhold else 0)


# ---------------------------------------------------------------------------
# instrumentation
# ---------------------------------------------------------------------------

def ca_prof_enable(on: bool, max_launches: int = 65536):
    _check("ca_prof_enable", load().ca_prof_enable(1 if on else 0, int(max_launches)))


def ca_prof_read(cls: int):
    """(launches, device ms, algorithmic flops, dropped) of one kernel class."""
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0)
    fl = ctypes.c_double(0)
    rc = load().ca_prof_read(int(cls), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl))
    if rc not in (0, 1):
        _check("ca_prof_read", rc)
    return n.value, ms.value, fl.value, rc == 1


def ca_launch_count(cls: int = -1) -> int:
    return int(load().ca_launch_count(int(cls)))


def ca_kernel_class_name(cls: int) -> str:
    return load().ca_kernel_class_name(int(cls)).decode()


def tslu_noalloc(A: torch.Tensor, tree: ca_tree_t, ipiv=None, dev_info=None, stream=None):
    """tslu with the library's static scratch instead of a workspace, for
    callers that cannot allocate device memory; see include/ca_gb300.h for the
    size limit and the rule that overlapping calls must be serialized."""
    L = load()
    L.tslu_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                               ctypes.POINTER(ca_tree_t), ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
    m, n, lda = _mat(A, "A")
    rc = L.tslu_noalloc(m, n, _ptr(A), lda, ctypes.byref(tree), _ptr(ipiv), _ptr(dev_info),
                        _stream(stream))
    _check("tslu_noalloc", rc)
    return ipiv, dev_info


def ca_gemm_mixed_workspace(m: int, n: int, k: int, slices: int, exact: bool) -> int:
    w = ctypes.c_size_t(0)
    _check("ca_gemm_mixed_workspace",
           load().ca_gemm_mixed_workspace(m, n, k, slices, 1 if exact else 0, ctypes.byref(w)))
    return w.value


def ca_gemm_minus_mixed(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, slices: int = 3,
                        exact: bool = False, work=None, dev_status=None, stream=None):
    """C -= A B on the tensor cores (split bf16 digits); returns dev_status."""
    m, k, lda = _mat(A, "A")
    k2, n, ldb = _mat(B, "B")
    mc, nc, ldc = _mat(C, "C")
    if k2 != k or mc != m or nc != n:
        raise ValueError("shape mismatch")
    if work is None:
        work = _buf(ca_gemm_mixed_workspace(m, n, k, slices, exact), A.device)
    if dev_status is None:
        dev_status = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = load().ca_gemm_minus_mixed(m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, slices,
                                    1 if exact else 0, _ptr(work), work.numel() * 8,
                                    _ptr(dev_status), _stream(stream))
    _check("ca_gemm_minus_mixed", rc)
    return dev_status


def ca_calu_mixed_workspace(m: int, n: int, b: int, tree: ca_tree_t, slices: int, exact: bool) -> int:
    w = ctypes.c_size_t(0)
    _check("ca_calu_mixed_workspace",
           load().ca_calu_mixed_workspace(m, n, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                          ctypes.byref(w)))
    return w.value


def calu_factor_mixed(A: torch.Tensor, b: int, tree: ca_tree_t, slices: int = 3, exact: bool = False,
                      ipiv=None, work=None, dev_info=None, stream=None):
    m, n, lda = _mat(A, "A")
    dev = A.device
    if ipiv is None:
        ipiv = torch.empty(max(1, min(m, n)), dtype=torch.int32, device=dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    if work is None:
        work = _buf(ca_calu_mixed_workspace(m, n, b, tree, slices, exact), dev)
    rc = load().calu_factor_mixed(m, n, _ptr(A), lda, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                  _ptr(ipiv), _ptr(work), work.numel() * 8, _ptr(dev_info), _stream(stream))
    _check("calu_factor_mixed", rc)
    return ipiv[: min(m, n)], dev_info


def _refine(refine) -> int:
    return REFINE[refine] if isinstance(refine, str) else int(refine)


def ca_gesv_mixed_workspace(n: int, nrhs: int, b: int, tree: ca_tree_t, slices: int, exact: bool,
                            refine="classic") -> int:
    w = ctypes.c_size_t(0)
    _check("ca_gesv_mixed_workspace",
           load().ca_gesv_mixed_workspace(n, nrhs, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                          _refine(refine), ctypes.byref(w)))
    return w.value


def calu_gesv_mixed(A: torch.Tensor, B: torch.Tensor, b: int, tree: ca_tree_t, slices: int = 3,
                    exact: bool = False, max_iter: int = 30, tol: float = 1e-14, refine="classic", LU=None,
                    X=None, ipiv=None, work=None, dev_info=None, iters=None, berr=None, stream=None):
    """Mixed-precision CALU + FP64 iterative refinement (refine: "classic",
    "gmres" or "auto").  Returns (X, iterations, backward error, dev_info);
    iterations (int32[1]) and backward error (float64[1]) are device tensors
    written on the stream (the call does not wait)."""
    n, n2, lda = _mat(A, "A")
    nb, nrhs, ldb = _mat(B, "B")
    dev = A.device
    if LU is None:
        LU = torch.empty((n, n), dtype=torch.float64, device=dev).t().contiguous().t()
    if X is None:
        X = torch.empty((n, nrhs), dtype=torch.float64, device=dev).t().contiguous().t()
    if ipiv is None:
        ipiv = torch.empty(max(1, n), dtype=torch.int32, device=dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    if iters is None:
        iters = torch.zeros(1, dtype=torch.int32, device=dev)
    if berr is None:
        berr = torch.zeros(1, dtype=torch.float64, device=dev)
    if work is None:
        work = _buf(ca_gesv_mixed_workspace(n, nrhs, b, tree, slices, exact, refine), dev)
    _, _, ldlu = _mat(LU, "LU")
    _, _, ldx = _mat(X, "X")
    rc = load().calu_gesv_mixed(n, nrhs, _ptr(A), lda, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                _refine(refine), _ptr(LU), ldlu, _ptr(ipiv), _ptr(B), ldb, _ptr(X), ldx,
                                _ptr(work), work.numel() * 8, max_iter, tol, _ptr(iters), _ptr(berr),
                                _ptr(dev_info), _stream(stream))
    _check("calu_gesv_mixed", rc)
    return X, iters, berr, dev_info


def ca_gels_mixed_workspace(m: int, n: int, nrhs: int, b: int, tree: ca_tree_t, slices: int, exact: bool):
    q = ctypes.c_size_t(0)
    w = ctypes.c_size_t(0)
    _check("ca_gels_mixed_workspace",
           load().ca_gels_mixed_workspace(m, n, nrhs, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                          ctypes.byref(q), ctypes.byref(w)))
    return q.value, w.value


def caqr_gels_mixed(A: torch.Tensor, B: torch.Tensor, b: int, tree: ca_tree_t, slices: int = 4,
                    exact: bool = True, max_iter: int = 10, tol: float = 1e-14, QR=None, qtree=None, X=None,
                    work=None, dev_info=None, iters=None, berr=None, stream=None):
    """Least squares by the reduced-precision CAQR + FP64 refinement.  Returns
    (X n x nrhs, iterations int32[1], stop measure float64[1], dev_info); the
    device tensors are written on the stream (the call does not wait)."""
    m, n, lda = _mat(A, "A")
    mb, nrhs, ldb = _mat(B, "B")
    dev = A.device
    qb, wb = ca_gels_mixed_workspace(m, n, nrhs, b, tree, slices, exact)
    if QR is None:
        QR = torch.empty((m, n), dtype=torch.float64, device=dev).t().contiguous().t()
    if qtree is None:
        qtree = _buf(qb, dev)
    if X is None:
        X = torch.empty((n, nrhs), dtype=torch.float64, device=dev).t().contiguous().t()
    if work is None:
        work = _buf(wb, dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    if iters is None:
        iters = torch.zeros(1, dtype=torch.int32, device=dev)
    if berr is None:
        berr = torch.zeros(1, dtype=torch.float64, device=dev)
    _, _, ldqr = _mat(QR, "QR")
    _, _, ldx = _mat(X, "X")
    rc = load().caqr_gels_mixed(m, n, nrhs, _ptr(A), lda, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                _ptr(QR), ldqr, _ptr(qtree), qtree.numel() * 8, _ptr(B), ldb, _ptr(X), ldx,
                                _ptr(work), work.numel() * 8, max_iter, tol, _ptr(iters), _ptr(berr),
                                _ptr(dev_info), _stream(stream))
    _check("caqr_gels_mixed", rc)
    return X, iters, berr, dev_info


def ca_caqr_mixed_workspace(m: int, n: int, b: int, tree: ca_tree_t, slices: int, exact: bool):
    q = ctypes.c_size_t(0)
    w = ctypes.c_size_t(0)
    _check("ca_caqr_mixed_workspace",
           load().ca_caqr_mixed_workspace(m, n, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                          ctypes.byref(q), ctypes.byref(w)))
    return q.value, w.value


def caqr_factor_mixed(A: torch.Tensor, b: int, tree: ca_tree_t, slices: int = 7, exact: bool = True,
                      qtree=None, work=None, dev_info=None, stream=None):
    """CAQR with the tree update on the tensor cores.  Returns (qtree, dev_info)."""
    m, n, lda = _mat(A, "A")
    dev = A.device
    qb, wb = ca_caqr_mixed_workspace(m, n, b, tree, slices, exact)
    if qtree is None:
        qtree = _buf(qb, dev)
    if work is None:
        work = _buf(wb, dev)
    if dev_info is None:
        dev_info = torch.zeros(2, dtype=torch.int32, device=dev)
    rc = load().caqr_factor_mixed(m, n, _ptr(A), lda, b, ctypes.byref(tree), slices, 1 if exact else 0,
                                  _ptr(qtree), qtree.numel() * 8, _ptr(work), work.numel() * 8,
                                  _ptr(dev_info), _stream(stream))
    _check("caqr_factor_mixed", rc)
    return qtree, dev_info


# ---------------------------------------------------------------------------
# batched factorizations
# ---------------------------------------------------------------------------

def ca_batched_plan(items, dtype: int):
    """Host plan of a batch: (plan bytes as a ctypes buffer, work bytes).
    ``items`` is a sequence of ca_batch_item_t."""
    arr = (ca_batch_item_t * max(1, len(items)))(*items)
    pb = ctypes.c_size_t(0)
    wb = ctypes.c_size_t(0)
    L = load()
    _check("ca_batched_plan", L.ca_batched_plan(len(items), arr, dtype, None, ctypes.byref(pb), ctypes.byref(wb)))
    plan = ctypes.create_string_buffer(pb.value)
    _check("ca_batched_plan", L.ca_batched_plan(len(items), arr, dtype, plan, ctypes.byref(pb), ctypes.byref(wb)))
    return plan, wb.value


def ca_batched_factor(plan_host, plan_dev: torch.Tensor, work: torch.Tensor, stream=None):
    rc = load().ca_batched_factor(ctypes.cast(plan_host, ctypes.c_void_p), _ptr(plan_dev), _ptr(work),
                                  work.numel() * work.element_size(), _stream(stream))
    _check("ca_batched_factor", rc)


class BatchedFactor:
    """Many CALU / CAQR factorizations in one persistent launch.

    ``mats``: 2-D column-major CUDA tensors, all float64 or all float32,
    factored in place.  ``ops[i]`` is "lu" or "qr"; ``bs[i]`` the panel width;
    ``trees[i]`` a ca_tree_t.  After ``run()``: ``ipiv(i)`` (LU), ``qtree(i)``
    (QR, the caqr_factor layout in the batch's type) and ``info(i)``.
    ``graph()`` captures the launch in a CUDA graph and returns it."""

    def __init__(self, mats, ops, bs, trees):
        if not mats:
            raise ValueError("empty batch")
        dt = mats[0].dtype
        if dt not in (torch.float64, torch.float32):
            raise TypeError("float64 or float32 matrices")
        self.dtype = CA_DTYPE_F64 if dt == torch.float64 else CA_DTYPE_F32
        dev = mats[0].device
        self.mats = list(mats)
        self.ops = list(ops)
        esz = 8 if dt == torch.float64 else 4
        ipiv_off, q_off = [], []
        ni, nq = 0, 0
        shapes = []
        for A, op, b, tree in zip(mats, ops, bs, trees):
            if A.dim() != 2 or A.dtype != dt or not A.is_cuda:
                raise TypeError("every matrix must be a 2-D CUDA tensor of the batch's dtype")
            m, n = A.shape
            if m > 0 and n > 0 and A.stride(0) != 1:
                raise ValueError("matrices must be column-major")
            lda = max(A.stride(1) if n > 1 else max(1, m), max(1, m))
            shapes.append((m, n, lda))
            ipiv_off.append(ni)
            q_off.append(nq)
            if op == "lu":
                ni += max(1, min(m, n))
            elif op == "qr":
                qb, _ = ca_caqr_workspace(m, n, b, tree) if n > 0 else (0, 0)
                nq += qb // 8
            else:
                raise ValueError("op must be 'lu' or 'qr'")
        self.ipiv_all = torch.zeros(max(1, ni), dtype=torch.int32, device=dev)
        self.qtree_all = torch.zeros(max(1, nq), dtype=dt, device=dev)
        self.info_all = torch.zeros(2 * len(mats), dtype=torch.int32, device=dev)
        self._ipiv_off, self._q_off = ipiv_off, q_off
        items = []
        for i, (A, op, b, tree) in enumerate(zip(mats, ops, bs, trees)):
            m, n, lda = shapes[i]
            it = ca_batch_item_t()
            it.op = CA_BATCH_CALU if op == "lu" else CA_BATCH_CAQR
            it.m, it.n, it.lda = m, n, lda
            it.A = A.data_ptr() if A.numel() > 0 else None
            it.ipiv = self.ipiv_all.data_ptr() + 4 * ipiv_off[i] if op == "lu" else None
            it.qtree = self.qtree_all.data_ptr() + esz * q_off[i] if op == "qr" else None
            it.info = self.info_all.data_ptr() + 8 * i
            it.b = int(b)
            it.tree = tree
            items.append(it)
        self.plan_host, wbytes = ca_batched_plan(items, self.dtype)
        raw = torch.frombuffer(bytearray(self.plan_host.raw), dtype=torch.uint8)
        self.plan_dev = raw.to(dev)
        self.work = torch.empty(max(1, (wbytes + 7) // 8), dtype=torch.float64, device=dev)

    def run(self, stream=None):
        ca_batched_factor(self.plan_host, self.plan_dev, self.work, stream)

    def graph(self):
        """A CUDA graph of the launch (replay with .replay())."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g

    def ipiv(self, i: int) -> torch.Tensor:
        m, n = self.mats[i].shape
        return self.ipiv_all[self._ipiv_off[i]: self._ipiv_off[i] + min(m, n)]

    def qtree(self, i: int) -> torch.Tensor:
        nxt = self._q_off[i + 1] if i + 1 < len(self._q_off) else self.qtree_all.numel()
        return self.qtree_all[self._q_off[i]: nxt]

    def info(self, i: int) -> torch.Tensor:
        return self.info_all[2 * i: 2 * i + 2]
