"""Batched and persistent execution on the GPU.

  * the persistent dataflow kernel and the per-step graph mode compute every tile identically,
    so their results agree bit for bit;
  * a batch of one circuit with many bitstrings, and a mixed batch of different circuits, sizes
    and partition counts, each match the state vector; every job's result is the same alone and
    in the mix (bit for bit: the tiles of one job never depend on the others);
  * bulk tensor updates (new bitstrings) are applied by the next run.
"""
import numpy as np
import pytest

from oracle import contract as oc
from oracle import costs as ocost
from oracle import greedy as og
from oracle import statevector as sv
from paper_2507_20667_gb300 import inputs as tni
from parity import TOL, amplitude_bitstring, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnsa():
    from paper_2507_20667_gb300 import tnsa as mod
    return mod


def oracle_amp(net):
    steps = og.greedy_steps(list(ocost.leaf_legs(net)), ocost.edge_dims(net))
    return oc.contract_scalar(net, steps)


def amps(tnsa, mant, e2):
    return np.array([complex(m) * 2.0 ** int(e) for m, e in zip(mant, e2)])


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_persistent_equals_graph_bitwise(tnsa, prec):
    circ, x = tni.cfg2()
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=4, iterations=300, seed=7,
                               position=net.qubit)
    out = {}
    for mode in ("persistent", "graph"):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_exec_mode(ctx, mode)
        m, e, info = tnsa.tn_contract(ctx, h, plan, prec)
        out[mode] = (m, e)
    assert out["persistent"] == out["graph"]


def test_one_circuit_many_bitstrings(tnsa):
    circ = tni.brickwork_1d(14, 10, seed=3)
    psi = sv.simulate(circ).reshape((2,) * 14)
    xs = [amplitude_bitstring(lambda y: psi[tuple(y)], 14, 900 + i, tni.random_bitstring)[0]
          for i in range(64)]
    nets = [tni.amplitude_tn(circ, x) for x in xs]
    hs = [tnsa.tn_build(n) for n in nets]
    plan = tnsa.tn_plan_create(hs[0], k=4, iterations=100, seed=1,
                               position=nets[0].qubit)
    ctx = tnsa.tn_ctx_create(0)
    b = tnsa.tn_batch_create(ctx, hs, [plan] * len(hs), "c64")
    tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, len(hs))
    assert (st == 0).all()
    got = amps(tnsa, mant, e2)
    for i, x in enumerate(xs):
        check(got[i], psi[tuple(x)], TOL["c64"], f"job {i}")
    # bulk update: flip every bit of the first 8 jobs and rerun
    n_t = nets[0].n_tensors
    jobs = np.repeat(np.arange(8, dtype=np.int32), 14)
    tensors = np.tile(np.arange(n_t - 14, n_t, dtype=np.int32), 8)
    flipped = [1 - x for x in xs[:8]]
    data = np.eye(2, dtype=np.complex128)[np.concatenate(flipped)]
    tnsa.tn_batch_set_tensors(b, jobs, tensors, data)
    tnsa.tn_batch_run(b)
    info = tnsa.tn_batch_last_info(b)
    assert 0 < info["h2d_bytes"] < 16384
    mant, e2, st = tnsa.tn_batch_results(b, len(hs))
    got2 = amps(tnsa, mant, e2)
    for i in range(8):
        check(got2[i], psi[tuple(flipped[i])], TOL["c64"], f"flipped job {i}")
    assert np.array_equal(got2[8:], got[8:])
    with pytest.raises(tnsa.TnError):
        tnsa.tn_batch_set_tensors(b, [len(hs)], [0], np.zeros(2, np.complex128))


def test_mixed_batch_alone_equals_mix(tnsa):
    specs = [(tni.brickwork_1d(10, 8, seed=11), 2), (tni.grid_2d(3, 4, 6, seed=12), 4),
             (tni.brickwork_1d(16, 9, seed=13), 8), (tni.grid_2d(4, 4, 5, seed=14), 2),
             (tni.ghz(12), 1)]
    nets, hs, plans, refs, nq = [], [], [], [], []
    for i, (circ, k) in enumerate(specs):
        for r in range(3):
            if i < 4:
                x, _, _ = amplitude_bitstring(lambda y: sv.amplitude(circ, y), circ.n_qubits, 70 * i + r,
                                              tni.random_bitstring)
            else:
                x = [r % 2] * 12
            net = tni.amplitude_tn(circ, x)
            h = tnsa.tn_build(net)
            pos = net.qubit if k > 1 else None
            plans.append(tnsa.tn_plan_create(h, k=k, iterations=60, seed=i, position=pos))
            nets.append(net)
            hs.append(h)
            refs.append(sv.amplitude(circ, x))
            nq.append(circ.n_qubits)
    ctx = tnsa.tn_ctx_create(0)
    for prec in ("c64", "c128"):
        mant, e2 = tnsa.tn_batch_contract(ctx, hs, plans, prec)
        mix = amps(tnsa, mant, e2)
        for i, ref in enumerate(refs):
            check(mix[i], ref, TOL[prec], f"{prec} job {i}")
        for i in (0, 4, 8, 13):
            m, e, _ = tnsa.tn_contract(ctx, hs[i], plans[i], prec)
            assert complex(m) * 2.0 ** e == mix[i]      # alone == in the mix, bit for bit


def test_batch_kernel_timing(tnsa):
    circ, x = tni.cfg1()
    nets = [tni.amplitude_tn(circ, tni.random_bitstring(10, i)) for i in range(32)]
    hs = [tnsa.tn_build(n) for n in nets]
    plan = tnsa.tn_plan_create(hs[0], k=1)
    ctx = tnsa.tn_ctx_create(0)
    b = tnsa.tn_batch_create(ctx, hs, [plan] * 32, "c64")
    for _ in range(3):
        tnsa.tn_batch_run(b)
    ms = tnsa.tn_batch_kernel_ms(b, 3)
    assert 0 < ms < 1000
    info = tnsa.tn_batch_last_info(b)
    # leaf conversion, one launch per program kind present, and the dataflow kernel when any step
    # is left outside the programs
    expect = 1 + (info["n_warp_progs"] > 0) + (info["n_local"] > 0) + \
        (info["n_gather"] + info["n_tile"] + info["n_dot"] > 0)
    assert info["launches"] == expect and info["flops"] > 0 and info["bytes"] > 0


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_subtree_programs_match_global_path(tnsa, prec):
    """CTA-resident subtree programs (shared memory) and the all-global step path agree."""
    circ, x = tni.cfg2()
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=4, iterations=300, seed=7,
                               position=net.qubit)
    ref = oracle_amp(net)
    res = {}
    for budget in (-1, 0, 16384):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_local_budget(ctx, budget)
        m, e, info = tnsa.tn_contract(ctx, h, plan, prec)
        res[budget] = (complex(m) * 2.0 ** e, info)
    assert res[-1][1]["n_local"] >= 1 and res[0][1]["n_local"] == 0
    assert res[16384][1]["n_local"] >= 1
    for budget in (-1, 0, 16384):
        check(res[budget][0], ref, TOL[prec], f"budget {budget}")


def test_context_freed_before_its_batch(tnsa):
    """Garbage collectors may free a context before the batches made from it: the context then
    lives on until its last batch is freed, and the batch keeps working meanwhile."""
    circ, x = tni.cfg1()
    h = tnsa.tn_build(tni.amplitude_tn(circ, x))
    plan = tnsa.tn_plan_create(h, k=1)
    ctx = tnsa.tn_ctx_create(0)
    b = tnsa.tn_batch_create(ctx, [h], [plan], "c64")
    ctx.close()
    tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, 1)
    assert st[0] == 0
    check(complex(mant[0]) * 2.0 ** int(e2[0]), sv.amplitude(circ, x), TOL["c64"])
    b.close()


@pytest.mark.parametrize("prec", ["c64", "bf16"])
def test_graph_replay_equals_direct_launches(tnsa, prec):
    """The default persistent path replays one recorded CUDA graph per run (reset, leaf conversion,
    programs, and per dependency phase the tensor-core pack and GEMM launches and the dataflow
    launch); issuing the same launches one by one gives the same bits."""
    circ, _ = tni.cfg3(small=True)
    nets = [tni.amplitude_tn(circ, tni.random_bitstring(20, 600 + i)) for i in range(16)]
    hs = [tnsa.tn_build(n) for n in nets]
    plan = tnsa.tn_plan_create(hs[0], k=8, iterations=100, seed=7, position=nets[0].qubit)
    out = {}
    for graph in (1, 0):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_config(ctx, graph_capture=graph)
        b = tnsa.tn_batch_create(ctx, hs, [plan] * len(hs), prec)
        for _ in range(3):
            tnsa.tn_batch_run(b)
        mant, e2, st = tnsa.tn_batch_results(b, len(hs))
        assert (st == 0).all()
        times = tnsa.tn_batch_kernel_times(b, 2)
        assert tnsa.tn_batch_kernel_ms(b, 3) > 0 and times["dataflow"] > 0
        if prec == "bf16":
            assert tnsa.tn_batch_last_info(b)["n_tc"] > 0 and times["tc_gemm"] > 0
        out[graph] = (mant.view(np.uint64).copy(), e2.copy())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_results_buffer_must_hold_every_job(tnsa):
    """tn_batch_results writes the result of every job of the batch: the binding refuses a count
    other than the batch's (a shorter host buffer would be overrun)."""
    circ, x = tni.cfg1()
    hs = [tnsa.tn_build(tni.amplitude_tn(circ, x)) for _ in range(3)]
    plan = tnsa.tn_plan_create(hs[0], k=1)
    ctx = tnsa.tn_ctx_create(0)
    b = tnsa.tn_batch_create(ctx, hs, [plan] * 3, "c64")
    tnsa.tn_batch_run(b)
    with pytest.raises(ValueError):
        tnsa.tn_batch_results(b, 2)
    mant, e2, st = tnsa.tn_batch_results(b)
    assert len(mant) == 3 and (st == 0).all()
    b.close()


def test_staged_updates_accumulate_and_alternate(tnsa):
    """Tensor updates are written into two pinned staging sets used in turn: several calls before
    one run accumulate (the run applies all of them), a rejected call stages nothing, and runs that
    alternate between the sets (each refilled only after its previous copy completed) keep giving
    the state vector's amplitudes."""
    circ = tni.brickwork_1d(12, 8, seed=4)
    psi = sv.simulate(circ).reshape((2,) * 12)
    rng = np.random.default_rng(31)
    x0 = [tni.random_bitstring(12, 700 + i) for i in range(6)]
    nets = [tni.amplitude_tn(circ, x) for x in x0]
    hs = [tnsa.tn_build(n) for n in nets]
    plan = tnsa.tn_plan_create(hs[0], k=2, iterations=50, seed=1, position=nets[0].qubit)
    ctx = tnsa.tn_ctx_create(0)
    b = tnsa.tn_batch_create(ctx, hs, [plan] * len(hs), "c64")
    tnsa.tn_batch_run(b)
    bras = tni.bra_ids(nets[0], 12)
    eye = np.eye(2, dtype=np.complex128)
    cur = [list(x) for x in x0]
    for rnd in range(5):
        # the new bitstrings of all jobs, staged in three calls (jobs 0-1, 2-3, 4-5)
        new = [rng.integers(0, 2, 12) for _ in range(6)]
        for lo in (0, 2, 4):
            jobs = np.repeat(np.arange(lo, lo + 2, dtype=np.int32), 12)
            tens = np.tile(np.asarray(bras, np.int32), 2)
            tnsa.tn_batch_set_tensors(b, jobs, tens, eye[np.concatenate(new[lo:lo + 2])])
        with pytest.raises(tnsa.TnError):   # a NaN entry: rejected, nothing staged
            tnsa.tn_batch_set_tensors(b, [0], [bras[0]], np.array([np.nan, 0.0], np.complex128))
        tnsa.tn_batch_run(b)
        cur = [list(x) for x in new]
        mant, e2, st = tnsa.tn_batch_results(b)
        assert (st == 0).all()
        got = amps(tnsa, mant, e2)
        for i, x in enumerate(cur):
            ref = psi[tuple(x)]
            if abs(ref) >= 1e-3 * 2.0 ** -6:
                check(got[i], ref, TOL["c64"], f"round {rnd} job {i}")
