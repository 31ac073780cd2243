"""GPU parity: the CUDA path (through the C ABI) against the complex128 oracle.

Every result is held to its plain relative error |a - a_ref| / |a_ref| (tests/parity.py):
complex128 1e-12 (against the state vector / oracle), complex64 1e-5, split-TF32 1e-5 and
split-BF16 1e-4 -- the bounds the workload definition states for single-amplitude results.
"""
import math

import numpy as np
import pytest

from oracle import contract as oc
from oracle import costs as ocost
from oracle import greedy as og
from oracle import statevector as sv
from paper_2507_20667_gb300 import inputs as tni
from parity import TOL, amplitude_bitstring, check, check_observable

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnsa():
    from paper_2507_20667_gb300 import tnsa as mod
    return mod


@pytest.fixture(scope="module")
def ctx(tnsa):
    return tnsa.tn_ctx_create(0)


def oracle_amp(net):
    steps = og.greedy_steps(list(ocost.leaf_legs(net)), ocost.edge_dims(net))
    return oc.contract_scalar(net, steps)


def gpu_amp(tnsa, ctx, net, plan=None, prec="c64", k=1, **kw):
    h = tnsa.tn_build(net)
    if plan is None:
        plan = tnsa.tn_plan_create(h, k=k, **kw)
    m, e, info = tnsa.tn_contract(ctx, h, plan, prec)
    return tnsa.amplitude(m, e), info


@pytest.mark.parametrize("prec", ["c128", "c64", "tf32", "bf16"])
def test_cfg1_all_precisions(tnsa, ctx, prec):
    circ, _ = tni.cfg1()
    x, ref, _ = amplitude_bitstring(lambda y: sv.amplitude(circ, y), 10, 1001, tni.random_bitstring)
    net = tni.amplitude_tn(circ, x)
    assert abs(oracle_amp(net) - ref) < 1e-13 * abs(ref)
    got, info = gpu_amp(tnsa, ctx, net, prec=prec)
    check(got, ref, TOL[prec])
    assert info["launches"] >= 1


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_closed_forms(tnsa, ctx, prec):
    n = 9
    g = tni.ghz(n)
    for bits, want in (([0] * n, 1 / math.sqrt(2)), ([1] * n, 1 / math.sqrt(2))):
        got, _ = gpu_amp(tnsa, ctx, tni.amplitude_tn(g, bits), prec=prec)
        check(got, want, TOL[prec], "GHZ")
    # an exactly zero amplitude has no relative error: its error is bounded on the scale 2^(-1/2)
    # of the nonzero ones
    got, _ = gpu_amp(tnsa, ctx, tni.amplitude_tn(g, [0, 1] + [0] * (n - 2)), prec=prec)
    assert abs(got) <= TOL[prec] / math.sqrt(2)
    circ = tni.brickwork_1d(8, 6, seed=31)
    for net in (tni.inverse_tn(circ), tni.norm_tn(circ)):
        got, _ = gpu_amp(tnsa, ctx, net, prec=prec, k=2, iterations=20,
                         position=net.qubit)
        check(got, 1.0, TOL[prec], "<0|C^-1 C|0> or <psi|psi>")
    zz = sv.zz_expectation(circ, 2, 6)
    got, _ = gpu_amp(tnsa, ctx, tni.zz_tn(circ, 2, 6), prec=prec)
    check_observable(got, zz, TOL[prec], 1.0, "<Z2 Z6>")


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_partition_and_order_invariance(tnsa, ctx, k):
    """The amplitude does not depend on the tree or the partitioning (Section 2.3)."""
    circ = tni.brickwork_1d(12, 10, seed=40)
    x, ref, _ = amplitude_bitstring(lambda y: sv.amplitude(circ, y), 12, 41, tni.random_bitstring)
    net = tni.amplitude_tn(circ, x)
    pos = net.qubit if k > 1 else None
    for mode in ("directed", "naive"):
        got, _ = gpu_amp(tnsa, ctx, net, prec="c128", k=k, mode=mode, iterations=30, seed=k,
                         position=pos)
        check(got, ref, TOL["c128"], mode)
        got, _ = gpu_amp(tnsa, ctx, net, prec="c64", k=k, mode=mode, iterations=30, seed=k,
                         position=pos)
        check(got, ref, TOL["c64"], mode)


@pytest.mark.parametrize("seed", range(6))
def test_random_networks_mixed_dims(tnsa, ctx, seed):
    """Non-power-of-two dimensions exercise the general (div/mod) index maps."""
    net = tni.random_network(14, 10, (1, 2, 3, 5, 6), seed=seed)
    ref = oracle_amp(net)
    for prec in ("c128", "c64"):
        got, _ = gpu_amp(tnsa, ctx, net, prec=prec)
        check(got, ref, TOL[prec], prec)


def test_random_tree_import(tnsa, ctx):
    """Arbitrary imported trees, with larger intermediates and the tiled kernel class."""
    net = tni.random_network(10, 12, (2, 3, 4), seed=77)
    ref = oracle_amp(net)
    rng = np.random.default_rng(5)
    n = net.n_tensors
    for trial in range(3):
        alive, steps, nxt = list(range(n)), [], n
        while len(alive) > 1:
            i, j = sorted(rng.choice(len(alive), 2, replace=False))
            a, b = alive[i], alive[j]
            steps.append((min(a, b), max(a, b)))
            alive = [t for t in alive if t not in (a, b)] + [nxt]
            nxt += 1
        h = tnsa.tn_build(net)
        plan = tnsa.tn_plan_import(h, steps)
        for prec in ("c128", "c64"):
            m, e, info = tnsa.tn_contract(ctx, h, plan, prec)
            check(tnsa.amplitude(m, e), ref, TOL[prec], f"tree {trial} {prec}")


@pytest.mark.parametrize("prec", ["c128", "c64", "tf32", "bf16"])
def test_cfg3_oracle_instance(tnsa, ctx, prec):
    """2D grid 4x5, depth 8, k = 8 partitions: against the 2^20 state vector."""
    circ, _ = tni.cfg3(small=True)
    x, ref, _ = amplitude_bitstring(lambda y: sv.amplitude(circ, y), 20, 1003, tni.random_bitstring)
    net = tni.amplitude_tn(circ, x)
    got, info = gpu_amp(tnsa, ctx, net, prec=prec, k=8, iterations=200, steps_per_temp=8, seed=7,
                        position=net.qubit)
    check(got, ref, TOL[prec])
    if prec in ("tf32", "bf16"):   # the dense fan-in steps run on the tensor cores
        assert info["n_tc"] > 0


def test_cfg2_full_size(tnsa, ctx):
    """24-qubit brickwork, depth 14, k = 4 SA partitions, complex64; the oracle contracts the
    same network along its own Greedy tree."""
    circ, _ = tni.cfg2()
    x, ref, _ = amplitude_bitstring(lambda y: oracle_amp(tni.amplitude_tn(circ, y)), 24, 1002,
                                    tni.random_bitstring)
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=4, iterations=2000, steps_per_temp=8, seed=7,
                               position=net.qubit)
    for prec in ("c64", "c128"):
        m, e, info = tnsa.tn_contract(ctx, h, plan, prec)
        check(tnsa.amplitude(m, e), ref, TOL[prec], prec)


def test_new_bitstring_reuploads_leaves(tnsa, ctx):
    circ, x = tni.cfg1()
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=1)
    y = 1 - np.asarray(x)
    n = circ.n_qubits
    for q in range(n):  # bra tensors are the last n tensors
        v = np.zeros(2, np.complex128)
        v[y[q]] = 1
        tnsa.tn_net_set_tensor(h, net.n_tensors - n + q, v)
    m, e, _ = tnsa.tn_contract(ctx, h, plan, "c128")
    check(tnsa.amplitude(m, e), sv.amplitude(circ, y), TOL["c128"])


def test_degenerate_networks(tnsa, ctx):
    class Net:
        pass
    # a single scalar tensor
    s = Net()
    s.degrees = np.array([0], np.int32)
    s.dims = np.zeros(0, np.int64)
    s.data = np.array([0.25, -0.5])
    s.edges = np.zeros((0, 4), np.int32)
    h = tnsa.tn_build(s)
    plan = tnsa.tn_plan_create(h, k=1)
    for prec in ("c128", "c64"):
        m, e, _ = tnsa.tn_contract(ctx, h, plan, prec)
        assert tnsa.amplitude(m, e) == complex(0.25, -0.5)
    # two disconnected closed components: the outer product of their amplitudes
    c1, c2 = tni.brickwork_1d(4, 3, seed=1), tni.brickwork_1d(5, 3, seed=2)
    n1 = tni.amplitude_tn(c1, [0, 1, 1, 0])
    n2 = tni.amplitude_tn(c2, [1, 1, 0, 0, 1])
    both = Net()
    both.tensors = n1.tensors + n2.tensors
    both.degrees = np.concatenate([n1.degrees, n2.degrees])
    both.dims = np.concatenate([n1.dims, n2.dims])
    both.data = np.concatenate([n1.data, n2.data])
    e2 = n2.edges.copy()
    e2[:, 0] += n1.n_tensors
    e2[:, 2] += n1.n_tensors
    both.edges = np.concatenate([n1.edges, e2])
    want = sv.amplitude(c1, [0, 1, 1, 0]) * sv.amplitude(c2, [1, 1, 0, 0, 1])
    h = tnsa.tn_build(both)
    for k in (1, 2, 3):
        plan = tnsa.tn_plan_create(h, k=k, iterations=10)
        m, e, _ = tnsa.tn_contract(ctx, h, plan, "c128")
        check(tnsa.amplitude(m, e), want, TOL["c128"], f"k={k}")
    # an open network is refused by the scalar entry point
    o = tni.random_network(5, 2, (2,), seed=1, n_open=1)
    h = tnsa.tn_build(o)
    plan = tnsa.tn_plan_create(h, k=1)
    with pytest.raises(tnsa.TnError) as ei:
        tnsa.tn_contract(ctx, h, plan, "c64")
    assert ei.value.status == tnsa.TN_EUNSUPPORTED


def test_budget_rejection(tnsa):
    ctx = tnsa.tn_ctx_create(0, hbm_budget_bytes=1024)
    net = tni.amplitude_tn(*tni.cfg1())
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=1)
    with pytest.raises(tnsa.TnError) as ei:
        tnsa.tn_contract(ctx, h, plan, "c64")
    assert ei.value.status == tnsa.TN_EBUDGET


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("shift", [-8, 8])
def test_power_of_two_scaling_is_load_bearing(tnsa, ctx, prec, shift):
    """Every leaf of cfg1 multiplied by 2^shift: the value is 2^(146 shift) times the amplitude,
    far outside the range of FP32 and of FP64 (2^-1168 or 2^1168), so only the per-step
    power-of-two scaling keeps the intermediates representable.  Scaling by powers of two is
    exact, so the mantissa is bit-identical to the unscaled run and the exponent moves by exactly
    146 shift; the unscaled value agrees with the oracle."""
    circ, x = tni.cfg1()
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=1)
    m0, e0, _ = tnsa.tn_contract(ctx, h, plan, prec)
    check(tnsa.amplitude(m0, e0), sv.amplitude(circ, x), TOL[prec])

    class Scaled:
        pass
    s = Scaled()
    s.degrees, s.dims, s.edges = net.degrees, net.dims, net.edges
    s.data = np.ldexp(np.asarray(net.data, np.float64), shift)
    hs = tnsa.tn_build(s)
    m1, e1, _ = tnsa.tn_contract(ctx, hs, tnsa.tn_plan_create(hs, k=1), prec)
    assert e1 - e0 == shift * net.n_tensors
    assert np.array([m1]).view(np.uint64).tolist() == np.array([m0]).view(np.uint64).tolist()


def test_rows_steps_with_odd_width(tnsa, ctx):
    """Mixed-dimension networks (dims 3 and 5) with every step global: the row kernel of the
    dataflow kernel runs steps of odd width N, where the paired 16-byte loads of B have a
    one-entry tail; compared with the oracle."""
    found = 0
    for seed in range(40):
        net = tni.random_network(12, 6, (3, 5), seed=seed)
        h = tnsa.tn_build(net)
        plan = tnsa.tn_plan_create(h, k=1)
        steps = tnsa.tn_plan_compile_steps(h, plan, "c64", 0)
        odd = [s for s in steps if s[0] == 0 and s[2] % 2 == 1 and s[2] > 1]
        if not odd:
            continue
        found += 1
        ref = oracle_amp(net)
        c = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_local_budget(c, 0)
        for prec in ("c64", "c128"):
            m, e, _ = tnsa.tn_contract(c, h, plan, prec)
            check(tnsa.amplitude(m, e), ref, TOL[prec], f"seed {seed} {prec}")
        if found == 4:
            break
    assert found >= 1


def _split_row_steps(geo):
    """Steps of a 256-thread block program that the narrow row kernel runs with 2 or 4 threads per
    row: not small enough for one warp (M N > 256 or M N K > 4096), N and K <= 16, and so few rows
    (R = 32 / NT per thread, NT = N rounded up to 4, 8 or 16) that at least half the threads would
    hold none.  Both operand orders are considered, since the program may swap A and B."""
    hits = []
    for kind, M, N, K, *_ in geo:
        for m, n in ((M, N), (N, M)):
            if n > 16 or K > 16 or not (m * n > 256 or m * n * K > 4096):
                continue
            nt = 4 if n <= 4 else 8 if n <= 8 else 16
            if 2 * -(-m // (32 // nt)) <= 256:
                hits.append((int(m), int(n), int(K)))
    return hits


def test_block_row_steps_shared_between_threads(tnsa, ctx):
    """Mixed-dimension networks (dims 3 and 5) that run entirely as subtree programs: their
    block-wide row steps with few rows share each row between 2 or 4 threads, and odd widths leave
    part of the last thread's columns empty.  Compared with the oracle in complex64 and
    complex128."""
    found = 0
    for seed in range(40):
        net = tni.random_network(12, 6, (3, 5), seed=seed)
        h = tnsa.tn_build(net)
        plan = tnsa.tn_plan_create(h, k=1)
        hits = [s for s in _split_row_steps(tnsa.tn_plan_compile_steps(h, plan, "c64", 0)) if s[1] % 2]
        progs = tnsa.tn_plan_compile_steps(h, plan, "c64", 64 * 1024)
        if not hits or not all(p[0] == 5 for p in progs):
            continue
        found += 1
        ref = oracle_amp(net)
        for prec in ("c64", "c128"):
            m, e, _ = tnsa.tn_contract(ctx, h, plan, prec)
            check(tnsa.amplitude(m, e), ref, TOL[prec], f"seed {seed} {prec} {hits}")
        if found == 6:
            break
    assert found >= 3


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_large_leaves_max_abs_across_slices(tnsa, ctx, prec):
    """Two vectors of 50000 entries (leaves above 64 entries are converted by blocks per slice of
    the leaf, whose max-abs values merge into one): their entries are about 2^60, except one near
    the end of each at 0.75 * 2^127, just below the largest entry the boundary accepts.  Scaled by
    the max-abs of the small entries alone, the product of the two large ones would overflow
    complex64; the true max-abs of the whole leaf keeps it finite, and a max-abs of 2^126 or more
    still gives a normal scale factor (the scale exponent stops at 126).  The dot product is
    compared with numpy on the stored values."""
    L = 50000
    rng = np.random.default_rng(11)
    big, small = 127, 60

    def vec():
        v = (rng.standard_normal(L) + 1j * rng.standard_normal(L)) * 2.0 ** small
        v[L - 7] = (0.75 + 0.5j) * 2.0 ** big
        return v

    class Dot:
        pass
    net = Dot()
    u, v = vec(), vec()
    net.degrees = np.array([1, 1], np.int32)
    net.dims = np.array([L, L], np.int64)
    net.edges = np.array([[0, 0, 1, 0]], np.int32)
    net.data = np.concatenate([u, v]).view(np.float64)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_import(h, [(0, 1)])
    m, e, _ = tnsa.tn_contract(ctx, h, plan, prec)
    m = complex(m)
    assert np.isfinite(m.real) and np.isfinite(m.imag)
    st = np.complex64 if prec == "c64" else np.complex128
    us, vs = u.astype(st).astype(np.complex128), v.astype(st).astype(np.complex128)

    def down(z):   # exact scaling by 2^-big, so that the products stay inside the float64 range
        return np.ldexp(z.real, -big) + 1j * np.ldexp(z.imag, -big)
    ref = np.dot(down(us), down(vs))
    got = complex(np.ldexp(m.real, int(e) - 2 * big), np.ldexp(m.imag, int(e) - 2 * big))
    check(got, ref, TOL[prec], f"{prec} dot of {L} entries")
