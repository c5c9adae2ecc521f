"""GPU parity of the batched factorizations (one persistent launch over many
uneven matrices, each with its own panel width and tree) against the CPU
oracle: CALU pivots exactly; every element of the factors, of every stored Y
and of every T within 1e-12 of its rounding scale (FP64; ``tests/parity.py``).
Also: zero pivots, empty and wide items, CUDA-graph replay equal to the plain
launch, and the benchmark's batch mix (sampled items against the oracle at
the same 1e-12, every item by its residual)."""
import numpy as np
import pytest

import oracle
from paper_1303_5837_gb300 import inputs
from tests.parity import check, lu_err, qr_err, qtree_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BIN, FLAT = 0, 1

# (op, m, n, b, leaf_rows, levels)
CASES = [
    ("lu", 96, 96, 32, 64, [(0, BIN)]),
    ("lu", 200, 200, 16, 64, [(2, BIN), (0, BIN)]),
    ("lu", 257, 257, 64, 128, [(0, FLAT)]),
    ("lu", 130, 130, 8, 32, [(4, FLAT), (0, BIN)]),
    ("lu", 512, 512, 64, 256, [(0, BIN)]),
    ("lu", 33, 33, 64, 64, [(0, BIN)]),
    ("lu", 1, 1, 4, 4, [(0, BIN)]),
    ("lu", 5, 3, 2, 2, [(0, BIN)]),
    ("lu", 40, 100, 16, 64, [(3, BIN), (0, FLAT)]),
    ("lu", 1000, 16, 16, 128, [(4, BIN), (0, BIN)]),
    ("lu", 8192, 64, 64, 256, [(0, BIN)]),
    ("lu", 3000, 128, 64, 128, [(2, FLAT), (0, BIN)]),
    ("lu", 700, 48, 48, 48, [(3, BIN), (2, FLAT), (0, BIN)]),
    ("qr", 96, 96, 32, 64, [(0, BIN)]),
    ("qr", 200, 200, 16, 64, [(2, BIN), (0, BIN)]),
    ("qr", 257, 257, 64, 128, [(0, FLAT)]),
    ("qr", 130, 130, 8, 32, [(4, FLAT), (0, BIN)]),
    ("qr", 512, 512, 64, 256, [(0, BIN)]),
    ("qr", 33, 33, 64, 64, [(0, BIN)]),
    ("qr", 1, 1, 4, 4, [(0, BIN)]),
    ("qr", 5, 3, 2, 2, [(0, BIN)]),
    ("qr", 1000, 16, 16, 128, [(4, BIN), (0, BIN)]),
    ("qr", 4096, 64, 64, 256, [(0, BIN)]),
    ("qr", 300, 32, 32, 64, [(2, FLAT), (0, BIN)]),
    ("qr", 3000, 128, 64, 128, [(0, BIN)]),
    ("qr", 700, 48, 48, 48, [(3, BIN), (2, FLAT), (0, BIN)]),
]


@pytest.fixture(scope="module")
def ca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1303_5837_gb300 as ca
    ca.load()
    return ca


def to_dev(A, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).to("cuda", dtype).t()


def run_batch(ca, cases, seed0, mats=None):
    hosts = mats or [inputs.gaussian(m, n, seed0 + i) for i, (_, m, n, *_r) in enumerate(cases)]
    devs = [to_dev(A) for A in hosts]
    bf = ca.BatchedFactor(devs, [c[0] for c in cases], [c[3] for c in cases],
                          [ca.make_tree(c[4], c[5]) for c in cases])
    bf.run()
    torch.cuda.synchronize()
    return hosts, devs, bf


def check_item(case, A, dev, bf, i, tol=1e-12, dtype=np.float64):
    op, m, n, b, L, lv = case
    got = dev.cpu().numpy()
    t = oracle.make_tree(L, lv)
    if op == "lu":
        LU_o, ipiv_o, info_o, nt = oracle.calu(A, b, t, dtype=dtype)
        assert nt == 0
        assert np.array_equal(bf.ipiv(i).cpu().numpy(), ipiv_o[: min(m, n)]), case
        check(lu_err(got, LU_o), tol, case)
        info = bf.info(i).cpu().tolist()
        assert info[0] == info_o, case
        if np.all(np.isfinite(LU_o)):   # a zero pivot's Inf / NaN is read by later panels
            assert info[1] == 0, case
    else:
        QR_o, T_o = oracle.caqr(A, b, t, dtype=dtype)
        check(qr_err(got, QR_o, b), tol, case)
        if min(m, n) > 0:
            check(qtree_err(bf.qtree(i).cpu().numpy(), T_o, QR_o, b, t, oracle.tree_counts), tol, case)
        assert bf.info(i).cpu().tolist() == [0, 0], case


def test_batched_fp64_matches_oracle(ca):
    hosts, devs, bf = run_batch(ca, CASES, 500)
    for i, case in enumerate(CASES):
        check_item(case, hosts[i], devs[i], bf, i)


def test_batched_zero_pivot_and_empty(ca):
    A = inputs.gaussian(64, 64, 3)
    A[:, 5] = 0.0            # U(5, 5) == 0: info = 6, factorization completes
    B = inputs.gaussian(64, 64, 4)
    B[:, 0] = 0.0
    cases = [("lu", 64, 64, 16, 32, [(0, BIN)]), ("lu", 64, 64, 8, 32, [(0, FLAT)]),
             ("qr", 64, 64, 16, 32, [(0, BIN)])]
    hosts, devs, bf = run_batch(ca, cases, 0, mats=[A, B, A.copy()])
    for i, case in enumerate(cases):
        check_item(case, hosts[i], devs[i], bf, i)
    assert bf.info(0).cpu().tolist()[0] == 6
    assert bf.info(1).cpu().tolist()[0] == 1
    # an empty item rides along and is left alone
    E = torch.zeros((0, 5), dtype=torch.float64, device="cuda")
    X = to_dev(inputs.gaussian(50, 20, 9))
    bf2 = ca.BatchedFactor([E, X], ["lu", "qr"], [4, 8], [ca.make_tree(8), ca.make_tree(16)])
    bf2.run()
    torch.cuda.synchronize()
    QR_o, _ = oracle.caqr(inputs.gaussian(50, 20, 9), 8, oracle.make_tree(16))
    check(qr_err(X.cpu().numpy(), QR_o, 8), 1e-12)


def test_batched_nonfinite_status(ca):
    A = inputs.gaussian(80, 80, 11)
    A[7, 3] = np.nan
    cases = [("lu", 80, 80, 16, 32, [(0, BIN)]), ("qr", 80, 80, 16, 32, [(0, BIN)])]
    _, _, bf = run_batch(ca, cases, 0, mats=[A, A.copy()])
    assert bf.info(0).cpu().tolist()[1] & 1
    assert bf.info(1).cpu().tolist()[1] & 1


def test_batched_graph_replay_equals_launch(ca):
    cases = CASES[:6] + CASES[13:19]
    hosts = [inputs.gaussian(c[1], c[2], 900 + i) for i, c in enumerate(cases)]
    ref = [to_dev(A) for A in hosts]
    bf_ref = ca.BatchedFactor(ref, [c[0] for c in cases], [c[3] for c in cases],
                              [ca.make_tree(c[4], c[5]) for c in cases])
    bf_ref.run()
    devs = [to_dev(A) for A in hosts]
    orig = [d.clone() for d in devs]
    bf = ca.BatchedFactor(devs, [c[0] for c in cases], [c[3] for c in cases],
                          [ca.make_tree(c[4], c[5]) for c in cases])
    g = bf.graph()             # runs once, then captures
    for d, o in zip(devs, orig):
        d.copy_(o)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(devs, ref):
        assert torch.equal(a, b)
    assert torch.equal(bf.ipiv_all, bf_ref.ipiv_all)
    assert torch.equal(bf.qtree_all, bf_ref.qtree_all)


def test_batched_plan_orders_largest_first(ca):
    from paper_1303_5837_gb300 import _binding as B
    import ctypes
    items = []
    for m, n in [(64, 64), (512, 512), (128, 128)]:
        it = B.ca_batch_item_t()
        it.op, it.m, it.n, it.lda, it.A, it.ipiv, it.info, it.b = 0, m, n, m, 16, 16, 16, 32
        it.tree = B.make_tree(64)
        items.append(it)
    plan, _ = B.ca_batched_plan(items, B.CA_DTYPE_F64)
    raw = plan.raw
    out = (B.ca_batch_item_t * 3).from_buffer_copy(raw[256: 256 + 3 * ctypes.sizeof(B.ca_batch_item_t)])
    assert [o.n for o in out] == [512, 128, 64]


@pytest.mark.slow
def test_batched_benchmark_mix(ca):
    """The benchmark's batch (square n in [32, 512], tall m in [256, 8192]
    with n in {16, 32, 64, 128}; CALU and CAQR of each) with the tuned
    shapes: 64 sampled items against the oracle, every item by its residual."""
    from paper_1303_5837_gb300 import tune
    mats, ops, bs, trees = tune.batch_workload(seed=77, count=256)
    devs = [to_dev(A) for A in mats]
    orig = [d.clone() for d in devs]
    bf = ca.BatchedFactor(devs, ops, bs, [ca.make_tree(L, lv) for L, lv in trees])
    bf.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for i in rng.choice(len(mats), 64, replace=False):
        op, b, (L, lv) = ops[i], bs[i], trees[i]
        check_item((op, *mats[i].shape, b, L, lv), mats[i], devs[i], bf, i)
    for i in range(len(mats)):
        A0, F = orig[i], devs[i]
        m, n = A0.shape
        if ops[i] == "lu":
            k = min(m, n)
            Lf = torch.tril(F[:, :k], -1) + torch.eye(m, k, dtype=F.dtype, device=F.device)
            U = torch.triu(F[:k, :])
            perm = torch.arange(m, device=F.device)
            for j, p in enumerate(bf.ipiv(i).cpu().tolist()):
                perm[[j, p - 1]] = perm[[p - 1, j]]
            res = torch.linalg.norm(A0[perm] - Lf @ U) / torch.linalg.norm(A0)
        else:
            R = torch.triu(F[:n])
            res = torch.linalg.norm(R.T @ R - A0.T @ A0) / torch.linalg.norm(A0) ** 2
        assert float(res) < 1e-13, (i, ops[i], m, n, float(res))


CASES32 = CASES + [("qr", 4096, 128, 128, 128, [(0, BIN)]), ("lu", 4096, 128, 128, 128, [(0, BIN)])]


def test_batched_fp32_matches_fp32_oracle(ca):
    """FP32 batch against the FP32 build of the oracle (pivot decisions in
    FP32 on both sides): pivots exactly wherever the oracle saw no near tie
    (runner-up within 1e-4); every factor, Y and T element within 1e-4 of its
    rounding scale (about 1700 FP32 unit roundoffs)."""
    hosts = [inputs.gaussian(c[1], c[2], 700 + i) for i, c in enumerate(CASES32)]
    devs = [to_dev(A, torch.float32) for A in hosts]
    bf = ca.BatchedFactor(devs, [c[0] for c in CASES32], [c[3] for c in CASES32],
                          [ca.make_tree(c[4], c[5]) for c in CASES32])
    bf.run()
    torch.cuda.synchronize()
    compared = 0
    for i, (op, m, n, b, L, lv) in enumerate(CASES32):
        got = devs[i].cpu().numpy()
        if op == "lu":
            LU_o, ipiv_o, info_o, nt = oracle.calu(hosts[i], b, oracle.make_tree(L, lv), dtype=np.float32)
            if nt:
                # a near tie decides a pivot by rounding: the GPU's own pivots
                # must still give a valid factorization
                perm, Lf, U = oracle.lu_unpack(got.astype(np.float64), bf.ipiv(i).cpu().numpy())
                A64 = hosts[i]
                assert np.linalg.norm(A64[perm] - Lf @ U) / np.linalg.norm(A64) < 1e-5, (op, m, n)
                continue
            compared += 1
            assert np.array_equal(bf.ipiv(i).cpu().numpy(), ipiv_o), (op, m, n)
            check(lu_err(got, LU_o), 1e-4, (op, m, n))
        else:
            t = oracle.make_tree(L, lv)
            QR_o, T_o = oracle.caqr(hosts[i], b, t, dtype=np.float32)
            compared += 1
            check(qr_err(got, QR_o, b), 1e-4, (op, m, n))
            check(qtree_err(bf.qtree(i).cpu().numpy(), T_o, QR_o, b, t, oracle.tree_counts), 1e-4, (op, m, n))
        assert bf.info(i).cpu().tolist() == [0, 0]
    assert compared >= len(CASES32) - 8


# (m, n, b, leaf_rows, levels, operator) -- CALU items with the 2D multilevel
# reduction operator of depth 1 and 2
OP_CASES = [
    (256, 256, 32, 64, [(0, BIN)], [(8, 16)]),
    (300, 300, 64, 128, [(2, BIN), (0, FLAT)], [(16, 32)]),
    (512, 512, 64, 256, [(0, BIN)], [(32, 64), (8, 16)]),
    (2000, 64, 64, 256, [(0, BIN)], [(16, 64), (4, 8)]),
    (777, 40, 40, 50, [(3, FLAT), (0, BIN)], [(8, 24)]),
    (100, 100, 16, 16, [(0, BIN)], [(16, 16)]),      # one inner panel per node: GEPP at the nodes
]


def test_batched_2d_operator_matches_oracle(ca):
    hosts = [inputs.gaussian(m, n, 1300 + i) for i, (m, n, *_r) in enumerate(OP_CASES)]
    devs = [to_dev(A) for A in hosts]
    bf = ca.BatchedFactor(devs, ["lu"] * len(OP_CASES), [c[2] for c in OP_CASES],
                          [ca.make_tree(c[3], c[4], c[5]) for c in OP_CASES])
    bf.run()
    torch.cuda.synchronize()
    for i, (m, n, b, L, lv, op) in enumerate(OP_CASES):
        LU_o, ipiv_o, info_o, nt = oracle.calu(hosts[i], b, oracle.make_tree(L, lv, op))
        assert nt == 0
        assert np.array_equal(bf.ipiv(i).cpu().numpy(), ipiv_o), (m, n, b, op)
        check(lu_err(devs[i].cpu().numpy(), LU_o), 1e-12, (m, n, b, op))
        assert bf.info(i).cpu().tolist() == [0, 0]
    # the operator changes the pivots of a genuine case
    plain = ca.BatchedFactor([to_dev(hosts[2])], ["lu"], [64], [ca.make_tree(256)])
    plain.run()
    torch.cuda.synchronize()
    assert not torch.equal(plain.ipiv(0), bf.ipiv(2))


def test_batched_2d_operator_rejected_for_qr(ca):
    t = ca.make_tree(64, op=[(8, 16)])
    A = to_dev(inputs.gaussian(128, 128, 1))
    with pytest.raises(ca.CaError):
        ca.caqr_factor(A, 32, t)
    with pytest.raises(ca.CaError):
        ca.BatchedFactor([A], ["qr"], [32], [t])
