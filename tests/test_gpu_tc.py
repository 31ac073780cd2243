"""Dense contraction steps on the tcgen05 tensor cores (BF16 or TF32 hi/lo split, FP32
accumulation).

trace(A B C) written as a closed network of three matrices: the first step A*B is a dense GEMM
(M = rows of A, N = columns of B, K = the shared leg), so in the split precisions it runs as
tensor-core tiles; the last step is the FP64 inner product with C.  Checked against the same
network in complex128 (CUDA cores) and against numpy.einsum.
"""
import numpy as np
import pytest

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
