"""The C-ABI library builds for sm_103a, loads, exports every symbol the
header declares, and rejects bad arguments on the host before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ca_gb300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_0-9]+)\s*\(", src)) - {"if", "sizeof"})


@pytest.fixture(scope="module")
def lib():
    from paper_1303_5837_gb300 import _binding
    return _binding.load()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for n in ["calu_factor", "caqr_factor", "tslu", "tsqr", "calu_getrs", "caqr_geqrs",
              "ca_calu_workspace", "ca_caqr_workspace", "ca_geqrs_workspace", "ca_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_abi():
    from paper_1303_5837_gb300 import _binding
    for name in declared_functions():
        if name != "ca_strerror":
            assert hasattr(_binding, name), name


def test_argument_errors_without_gpu(lib):
    from paper_1303_5837_gb300 import _binding as B
    t = B.make_tree(128)
    size = ctypes.c_size_t()
    assert lib.ca_calu_workspace(-1, 10, 64, ctypes.byref(t), ctypes.byref(size)) == -1
    assert lib.ca_calu_workspace(10, -1, 64, ctypes.byref(t), ctypes.byref(size)) == -2
    assert lib.ca_calu_workspace(10, 10, 0, ctypes.byref(t), ctypes.byref(size)) == -3
    small = B.make_tree(32)   # leaf_rows < b
    assert lib.ca_calu_workspace(100, 100, 64, ctypes.byref(small), ctypes.byref(size)) == -4
    assert lib.ca_calu_workspace(1024, 1024, 64, ctypes.byref(t), ctypes.byref(size)) == 0
    assert size.value > 0
    q = ctypes.c_size_t()
    assert lib.ca_caqr_workspace(10, 20, 8, ctypes.byref(t), ctypes.byref(q), ctypes.byref(size)) == -2
    assert lib.ca_caqr_workspace(1024, 512, 64, ctypes.byref(t), ctypes.byref(q), ctypes.byref(size)) == 0
    # bad arguments are reported before anything touches the (null) stream
    assert lib.calu_factor(-1, 4, None, 4, 4, ctypes.byref(t), None, None, 0, None, None) == -1
    assert lib.calu_factor(4, 4, None, 4, 4, ctypes.byref(t), None, None, 0, None, None) == -3
    assert lib.calu_factor(8, 8, ctypes.c_void_p(16), 4, 4, ctypes.byref(t), None, None, 0, None, None) == -4
    assert lib.calu_getrs(-3, 1, None, 1, None, None, 1, None, 0, None) == -1
    # the solve workspace is the caller's: too small is refused before any launch
    assert lib.calu_getrs(300, 1, ctypes.c_void_p(256), 300, ctypes.c_void_p(256), ctypes.c_void_p(256), 300,
                          ctypes.c_void_p(256), 4, None) == -1001
    assert lib.ca_getrs_workspace(300, 1, ctypes.byref(size)) == 0 and 0 < size.value <= 4096
    assert lib.ca_getrs_workspace(-1, 1, ctypes.byref(size)) == -1
    assert lib.caqr_factor(4, 8, None, 4, 4, ctypes.byref(t), None, 0, None, 0, None, None) == -2
    assert lib.ca_strerror(-1001).decode().startswith("workspace")
    wide = B.make_tree(512)
    assert lib.ca_calu_workspace(4096, 4096, 256, ctypes.byref(wide), ctypes.byref(size)) == -1002
    # solve status: NULL workspace or result pointers are argument errors
    flag = ctypes.c_int(7)
    assert lib.ca_solve_status(None, ctypes.byref(flag), None) == -1
    assert lib.ca_solve_status(ctypes.c_void_p(256), None, None) == -2
    # refinement: an unknown correction method is refused (argument 7 of the query)
    assert lib.ca_gesv_mixed_workspace(512, 1, 64, ctypes.byref(t), 4, 1, 9, ctypes.byref(size)) == -7
    assert lib.ca_gesv_mixed_workspace(512, 1, 64, ctypes.byref(t), 4, 1, 2, ctypes.byref(size)) == 0
    classic = ctypes.c_size_t()
    assert lib.ca_gesv_mixed_workspace(512, 1, 64, ctypes.byref(t), 4, 1, 0, ctypes.byref(classic)) == 0
    assert size.value > classic.value      # the GMRES correction's Krylov basis
    # least squares: m < n, a bad tree, too many digits are argument errors
    q = ctypes.c_size_t()
    assert lib.ca_gels_mixed_workspace(10, 20, 1, 8, ctypes.byref(t), 4, 1, ctypes.byref(q),
                                       ctypes.byref(size)) == -2
    assert lib.ca_gels_mixed_workspace(1000, 300, 1, 64, ctypes.byref(B.make_tree(32)), 4, 1, ctypes.byref(q),
                                       ctypes.byref(size)) == -5
    assert lib.ca_gels_mixed_workspace(1000, 300, 1, 64, ctypes.byref(t), 9, 1, ctypes.byref(q),
                                       ctypes.byref(size)) == -6
    assert lib.ca_gels_mixed_workspace(1000, 300, 2, 64, ctypes.byref(t), 4, 1, ctypes.byref(q),
                                       ctypes.byref(size)) == 0 and q.value > 0 and size.value > 0


def test_workspace_matches_tree_counts(lib):
    """qtree bytes = sum over panels of (leaves + merges) b^2 doubles, the
    layout the header documents (counts from the oracle's tree)."""
    import oracle
    from paper_1303_5837_gb300 import _binding as B
    for (m, n, b, L, lv) in [(1000, 300, 32, 64, [(2, 0), (0, 0)]), (777, 64, 64, 128, [(3, 1), (0, 0)]),
                             (4096, 128, 64, 256, [(4, 0), (4, 0), (0, 1)])]:
        qb, _ = B.ca_caqr_workspace(m, n, b, B.make_tree(L, lv))
        assert qb == 8 * oracle.caqr_tcount(m, n, b, oracle.make_tree(L, lv))


def test_batched_plan_checks_without_gpu(lib):
    """The batched plan is host data: validation, sizes and the LPT order
    need no GPU; a launch with a foreign buffer is refused before any work."""
    from paper_1303_5837_gb300 import _binding as B
    pb, wb = ctypes.c_size_t(), ctypes.c_size_t()

    def item(op=0, m=100, n=100, b=32, L=64, levels=((0, 0),)):
        it = B.ca_batch_item_t()
        it.op, it.m, it.n, it.lda, it.b = op, m, n, max(m, 1), b
        it.A, it.ipiv, it.qtree, it.info = 256, 256, 256, 256
        it.tree = B.make_tree(L, levels)
        return it

    def plan(items, dtype=B.CA_DTYPE_F64):
        arr = (B.ca_batch_item_t * max(1, len(items)))(*items)
        return lib.ca_batched_plan(len(items), arr, dtype, None, ctypes.byref(pb), ctypes.byref(wb))

    assert lib.ca_batched_plan(-1, None, 0, None, ctypes.byref(pb), ctypes.byref(wb)) == -1
    assert lib.ca_batched_plan(1, None, 0, None, ctypes.byref(pb), ctypes.byref(wb)) == -2
    assert plan([item()], dtype=7) == -3
    assert plan([item(op=5)]) == B.CA_ERR_BATCH_ITEM
    assert plan([item(op=1, m=10, n=20)]) == B.CA_ERR_BATCH_ITEM         # QR needs m >= n
    assert plan([item(L=16)]) == B.CA_ERR_BATCH_ITEM                      # leaf_rows < b
    assert plan([item(b=96, L=128)]) == B.CA_ERR_UNSUPPORTED              # > 64 with an update
    # FP64 binary merge of two 128-wide candidate sets (257 x 128) exceeds shared memory ...
    assert plan([item(op=1, m=4096, n=128, b=128, L=128)]) == B.CA_ERR_UNSUPPORTED
    # ... FP32 holds it
    assert plan([item(op=1, m=4096, n=128, b=128, L=128)], dtype=B.CA_DTYPE_F32) == 0
    assert plan([item(), item(op=1, m=3000, n=64, b=64, L=256)]) == 0
    assert pb.value == 256 + 2 * ctypes.sizeof(B.ca_batch_item_t)
    assert wb.value > 256
    bogus = ctypes.create_string_buffer(256)
    assert lib.ca_batched_factor(bogus, None, None, 0, None) == -1


def test_corrupted_tree_is_rejected_on_the_host(lib):
    """Fault injection on the host: a corrupted tree description (no levels,
    too many levels, an unknown merge style, a zero fan-in below the top, a
    NULL pointer, leaves narrower than the panel) is reported as a bad tree
    argument by every query before anything is enqueued."""
    from paper_1303_5837_gb300 import _binding as B
    size, q = ctypes.c_size_t(), ctypes.c_size_t()

    def corrupt():
        out = []
        t = B.make_tree(128); t.nlevels = 0; out.append(t)
        t = B.make_tree(128); t.nlevels = 9; out.append(t)
        t = B.make_tree(128); t.style[0] = 7; out.append(t)
        out.append(B.make_tree(128, [(0, 0), (0, 0)]))
        out.append(B.make_tree(32))   # leaf rows < b = 64
        return out

    for t in corrupt() + [None]:
        ref = ctypes.byref(t) if t is not None else None
        assert lib.ca_calu_workspace(4096, 256, 64, ref, ctypes.byref(size)) == -4
        assert lib.ca_caqr_workspace(4096, 256, 64, ref, ctypes.byref(q), ctypes.byref(size)) == -4
        assert lib.ca_geqrs_workspace(4096, 256, 1, 64, ref, ctypes.byref(size)) == -5
    # a deep but well-formed tree is accepted (one leaf per row, 26 binary rounds)
    deep = B.make_tree(1)
    assert lib.ca_calu_workspace(1 << 26, 1, 1, ctypes.byref(deep), ctypes.byref(size)) == 0
