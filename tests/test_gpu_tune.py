"""Execution configurations and the autotuner.

Every configuration of the program compiler -- warp programs, block programs, large programs on
or off, no programs at all -- executes the same contraction tree, so the amplitudes agree with the
state vector within the complex64 tolerance in every one of them; the autotuner times each
candidate on the batch, keeps the fastest in the context, and that configuration is the one the
context then reports.
"""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2507_20667_gb300 import inputs as tni
from parity import TOL, amplitude_bitstring, check_all

pytestmark = pytest.mark.gpu

N_Q = 16


@pytest.fixture(scope="module")
def tnsa():
    from paper_2507_20667_gb300 import tnsa as mod
    return mod


@pytest.fixture(scope="module")
def batch_inputs(tnsa):
    circ = tni.brickwork_1d(N_Q, 10, seed=11)
    psi = sv.simulate(circ).reshape((2,) * N_Q)
    xs = [amplitude_bitstring(lambda y: psi[tuple(y)], N_Q, 300 + i, tni.random_bitstring)[0]
          for i in range(24)]
    nets = [tni.amplitude_tn(circ, x) for x in xs]
    hs = [tnsa.tn_build(n) for n in nets]
    plan = tnsa.tn_plan_create(hs[0], k=4, iterations=100, seed=3,
                               position=nets[0].qubit)
    ref = np.array([psi[tuple(x)] for x in xs])
    return hs, plan, ref


def _check(got, ref):
    check_all(got, ref, TOL["c64"])


def _run(tnsa, ctx, hs, plan):
    b = tnsa.tn_batch_create(ctx, hs, [plan] * len(hs), "c64")
    tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, len(hs))
    assert (st == 0).all()
    info = tnsa.tn_batch_last_info(b)
    b.close()
    return mant * np.ldexp(1.0, e2), info


@pytest.mark.parametrize("cfg", [dict(big_programs=0), dict(warp_programs=0), dict(big_programs=0, warp_programs=0),
                                 dict(local_budget=0), dict(local_budget=24576)])
def test_configurations_agree_with_state_vector(tnsa, batch_inputs, cfg):
    hs, plan, ref = batch_inputs
    ctx = tnsa.tn_ctx_create(0)
    tnsa.tn_ctx_set_config(ctx, **cfg)
    got, info = _run(tnsa, ctx, hs, plan)
    _check(got, ref)
    if cfg.get("warp_programs") == 0 or cfg.get("local_budget") == 0:
        assert info["n_warp_progs"] == 0
    if cfg.get("local_budget") == 0:
        assert info["n_local"] == 0


def test_autotune_keeps_the_fastest(tnsa, batch_inputs):
    hs, plan, ref = batch_inputs
    ctx = tnsa.tn_ctx_create(0)
    best, ms, cands = tnsa.tn_ctx_autotune(ctx, hs, [plan] * len(hs), "c64", runs=3)
    ok = [c for c in cands if c > 0]
    assert len(ok) >= 2 and ms == pytest.approx(min(ok))
    assert tnsa.tn_ctx_get_config(ctx) == best
    got, _ = _run(tnsa, ctx, hs, plan)
    _check(got, ref)


def _run_bits(tnsa, ctx, hs, plan):
    b = tnsa.tn_batch_create(ctx, hs, [plan] * len(hs), "c64")
    tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, len(hs))
    b.close()
    assert (st == 0).all()
    return mant, e2


@pytest.mark.parametrize("budget", [0, 4096, -1])
def test_rows_chains_are_bit_identical(tnsa, batch_inputs, budget):
    """A chain of ROWS steps run in one block with the tensor kept in shared memory computes the
    same arithmetic in the same order as the separate steps, and carries the per-step scale
    exponents unchanged: mantissas and exponents agree bit for bit."""
    hs, plan, ref = batch_inputs
    if budget >= 0:
        assert tnsa.tn_plan_compile_stats(hs[0], plan, "c64", budget)["n_chained"] > 0
    out = []
    for chains in (1, 0):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_config(ctx, local_budget=budget, rows_chains=chains)
        out.append(_run_bits(tnsa, ctx, hs, plan))
    (m1, e1), (m0, e0) = out
    assert np.array_equal(e1, e0)
    assert np.array_equal(m1.view(np.uint64), m0.view(np.uint64))
    _check(m1 * np.ldexp(1.0, e1), ref)


def test_critical_path_schedule_is_bit_identical(tnsa, batch_inputs):
    """The critical-path-first work order (path sums of Eq. 3.4) changes only when tiles run, not
    what they compute: the results equal the level order's bit for bit."""
    hs, plan, ref = batch_inputs
    out = []
    for sched in (0, 1):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_config(ctx, schedule=sched, local_budget=4096)
        out.append(_run_bits(tnsa, ctx, hs, plan))
    (m0, e0), (m1, e1) = out
    assert np.array_equal(e0, e1) and np.array_equal(m0.view(np.uint64), m1.view(np.uint64))
    _check(m1 * np.ldexp(1.0, e1), ref)
