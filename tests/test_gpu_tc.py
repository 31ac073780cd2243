"""Dense contraction steps on the tcgen05 tensor cores (BF16 or TF32 hi/lo split, FP32
accumulation).

trace(A B C) written as a closed network of three matrices: the first step A*B is a dense GEMM
(M = rows of A, N = columns of B, K = the shared leg), so in the split precisions it runs as
tensor-core tiles; the last step is the FP64 inner product with C.  Checked against the same
network in complex128 (CUDA cores) and against numpy.einsum.
"""
import numpy as np
import pytest

from parity import TOL, check_scaled

pytestmark = pytest.mark.gpu


class _Trace:
    """transposed_a: A is stored K x I, so the GEMM's row index (I) is A's contiguous one."""
    def __init__(self, I, K, J, seed, transposed_a=False):
        rng = np.random.default_rng(seed)
        def rnd(*s):
            return (rng.standard_normal(s) + 1j * rng.standard_normal(s)) / np.sqrt(2)
        self.A, self.B, self.C = rnd(I, K), rnd(K, J), rnd(J, I)
        a_store = self.A.T.copy() if transposed_a else self.A
        self.tensors = [a_store, self.B, self.C]
        self.degrees = np.array([2, 2, 2], np.int32)
        self.dims = np.array([K, I, K, J, J, I] if transposed_a else [I, K, K, J, J, I], np.int64)
        self.data = np.concatenate([t.ravel() for t in self.tensors]).view(np.float64)
        if transposed_a:   # A axis 0 - B axis 0 (K); B axis 1 - C axis 0 (J); C axis 1 - A axis 1 (I)
            self.edges = np.array([[0, 0, 1, 0], [1, 1, 2, 0], [2, 1, 0, 1]], np.int32)
        else:              # A axis 1 - B axis 0 (K); B axis 1 - C axis 0 (J); C axis 1 - A axis 0 (I)
            self.edges = np.array([[0, 1, 1, 0], [1, 1, 2, 0], [2, 1, 0, 0]], np.int32)

    def exact(self):
        return complex(np.einsum("ik,kj,ji->", self.A, self.B, self.C))


@pytest.fixture(scope="module")
def tnsa():
    from paper_2507_20667_gb300 import tnsa as mod
    return mod


@pytest.mark.parametrize("shape", [(256, 64, 256), (200, 40, 100), (128, 512, 96), (64, 16, 32),
                                   (256, 64, 256, True), (136, 48, 72, True)])
def test_tc_gemm_matches_c128(tnsa, shape):
    """Both gather orders of the operand tiles: k contiguous in A, and (transposed A) the row
    index contiguous in A; B always has its column index contiguous."""
    net = _Trace(*shape[:3], seed=sum(shape[:3]), transposed_a=len(shape) > 3)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_import(h, [(0, 1), (2, 3)])
    ref = net.exact()
    res = {}
    for prec in ("c128", "c64", "bf16", "tf32"):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_local_budget(ctx, 0)
        m, e, info = tnsa.tn_contract(ctx, h, plan, prec)
        res[prec] = (complex(m) * 2.0 ** e, info)
    assert res["bf16"][1]["n_tc"] == 1 and res["tf32"][1]["n_tc"] == 1 and res["c64"][1]["n_tc"] == 0
    assert abs(res["c128"][0] - ref) <= 1e-12 * abs(ref)
    assert abs(res["c64"][0] - ref) <= 1e-5 * abs(ref)
    assert abs(res["bf16"][0] - ref) <= 1e-4 * abs(ref), (res["bf16"][0], ref)
    # three TF32 products carry about 21 bits: the complex64 tolerance
    assert abs(res["tf32"][0] - ref) <= 1e-5 * abs(ref), (res["tf32"][0], ref)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_persistent_equals_graph(tnsa, prec):
    net = _Trace(256, 96, 192, seed=5)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_import(h, [(0, 1), (2, 3)])
    out = {}
    for mode in ("persistent", "graph"):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_local_budget(ctx, 0)
        tnsa.tn_ctx_set_exec_mode(ctx, mode)
        m, e, info = tnsa.tn_contract(ctx, h, plan, prec)
        out[mode] = (m, e)
        assert info["n_tc"] == 1
    assert out["persistent"] == out["graph"]


def test_tc_in_a_batch(tnsa):
    """Several GEMM-bearing jobs in one persistent launch (each block holds its TMEM accumulator
    across tiles of different jobs)."""
    nets = [_Trace(192, 64, 160, seed=s) for s in range(6)]
    hs = [tnsa.tn_build(n) for n in nets]
    plans = [tnsa.tn_plan_import(h, [(0, 1), (2, 3)]) for h in hs]
    ctx = tnsa.tn_ctx_create(0)
    tnsa.tn_ctx_set_local_budget(ctx, 0)
    b = tnsa.tn_batch_create(ctx, hs, plans, "bf16")
    for _ in range(2):
        tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, len(hs))
    assert (st == 0).all()
    for i, n in enumerate(nets):
        ref = n.exact()
        assert abs(complex(mant[i]) * 2.0 ** int(e2[i]) - ref) <= 1e-4 * abs(ref)


class _Bilinear:
    """u^T (A B) v with A [I, K], B [K, J] and vectors u [I], v [J]: with one-hot u and v the
    network's value is one element C[i, j] of the product, which the engine computes as a dense
    tensor-core step followed by two exact selections (sums with a single nonzero term)."""
    def __init__(self, I, K, J, seed):
        rng = np.random.default_rng(seed)
        def rnd(*s):
            return (rng.standard_normal(s) + 1j * rng.standard_normal(s)) / np.sqrt(2)
        self.A, self.B = rnd(I, K), rnd(K, J)
        self.I, self.J = I, J
        u, v = np.zeros(I, complex), np.zeros(J, complex)
        u[0] = v[0] = 1
        self.tensors = [self.A, self.B, u, v]
        self.degrees = np.array([2, 2, 1, 1], np.int32)
        self.dims = np.array([I, K, K, J, I, J], np.int64)
        self.data = np.concatenate([t.ravel() for t in self.tensors]).view(np.float64)
        # A axis 1 - B axis 0 (K); A axis 0 - u (I); B axis 1 - v (J)
        self.edges = np.array([[0, 1, 1, 0], [0, 0, 2, 0], [1, 1, 3, 0]], np.int32)


def _edge_samples(extent, tile, rng, extra):
    """Indices on both sides of every tile boundary, the last index, and random ones."""
    s = {0, extent - 1}
    for b in range(tile, extent, tile):
        s.update((b - 1, b))
    s.update(int(i) for i in rng.integers(0, extent, extra))
    return sorted(s)


@pytest.mark.parametrize("shape,tile", [((200, 40, 100), 0), ((200, 40, 100), 64), ((136, 48, 72), 128),
                                        ((136, 48, 60), 0), ((1024, 512, 1024), 0)])
@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_gemm_elementwise(tnsa, shape, tile, prec):
    """Elements of the tensor-core product C = A B at sampled (i, j) covering every 128-row and
    64-column tile edge and the ragged tails (M, N, K not multiples of 128, 64 and 32), each within
    1e-4 (BF16 split) or 1e-5 (TF32 split) of max |C| against numpy complex128; output tiles of 64
    and of 128 complex columns (tile 0: 64 when N <= 64)."""
    I, K, J = shape
    net = _Bilinear(I, K, J, seed=I + K + J)
    C = net.A @ net.B
    scale = np.abs(C).max()
    rng = np.random.default_rng(I * J)
    rows = _edge_samples(I, 128, rng, 3)
    cols = _edge_samples(J, 64, rng, 3)
    # every sampled row with a random column and every sampled column with a random row, plus the
    # four corners of the product
    pairs = sorted({(i, int(rng.integers(0, J))) for i in rows} | {(int(rng.integers(0, I)), j) for j in cols}
                   | {(0, 0), (0, J - 1), (I - 1, 0), (I - 1, J - 1)})
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_import(h, [(0, 1), (2, 4), (3, 5)])
    steps = tnsa.tn_plan_compile_steps(h, plan, prec, 0)
    assert steps[0, 0] == 4, "the product must run as a tensor-core step"
    ctx = tnsa.tn_ctx_create(0)
    tnsa.tn_ctx_set_config(ctx, local_budget=0, tc_tile_n=tile)
    b = tnsa.tn_batch_create(ctx, [h] * len(pairs), [plan] * len(pairs), prec)
    jobs, tens, data = [], [], []
    for q, (i, j) in enumerate(pairs):
        u, v = np.zeros(I, complex), np.zeros(J, complex)
        u[i] = v[j] = 1
        jobs += [q, q]
        tens += [2, 3]
        data += [u, v]
    tnsa.tn_batch_set_tensors(b, jobs, tens, np.concatenate(data))
    tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, len(pairs))
    assert (st == 0).all()
    got = mant * np.ldexp(1.0, e2)
    want = np.array([C[i, j] for i, j in pairs])
    check_scaled(got, want, scale, TOL[prec], f"{len(pairs)} elements of C")


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_long_k_does_not_drift(tnsa, prec):
    """A long shared index (K = 16384: 1024 BF16 or 2048 TF32 k-blocks) is accumulated in segments
    whose partial sums are added in FP32 on the CUDA cores, so the tensor cores' non-nearest
    accumulation cannot shrink the product systematically: the mean radial error of sampled
    elements, Re((got - want) conj(want)) / |want|^2, stays at the size of one segment's drift
    (below 5e-6), where a single accumulator over all of K drifted by -1e-4 (BF16) and -2e-4
    (TF32)."""
    I, K, J = 128, 16384, 128
    net = _Bilinear(I, K, J, seed=K)
    C = net.A @ net.B
    rng = np.random.default_rng(K)
    pairs = [(int(rng.integers(0, I)), int(rng.integers(0, J))) for _ in range(64)]
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_import(h, [(0, 1), (2, 4), (3, 5)])
    ctx = tnsa.tn_ctx_create(0)
    tnsa.tn_ctx_set_config(ctx, local_budget=0)
    b = tnsa.tn_batch_create(ctx, [h] * len(pairs), [plan] * len(pairs), prec)
    jobs, tens, data = [], [], []
    for q, (i, j) in enumerate(pairs):
        u, v = np.zeros(I, complex), np.zeros(J, complex)
        u[i] = v[j] = 1
        jobs += [q, q]
        tens += [2, 3]
        data += [u, v]
    tnsa.tn_batch_set_tensors(b, jobs, tens, np.concatenate(data))
    tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, len(pairs))
    assert (st == 0).all()
    assert tnsa.tn_batch_last_info(b)["n_tc"] == len(pairs)
    got = mant * np.ldexp(1.0, e2)
    want = np.array([C[i, j] for i, j in pairs])
    radial = np.real((got - want) * np.conj(want)) / np.abs(want) ** 2
    assert abs(radial.mean()) < 5e-6, f"mean radial error {radial.mean():.3e}"
    check_scaled(got, want, np.abs(C).max(), TOL[prec], f"{len(pairs)} elements of C, K = {K}")
