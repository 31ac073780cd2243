"""Failure detection on the GPU without a GPU fault: bounded device-side waits.

The persistent dataflow kernel waits for the steps producing a tile's operands with a bounded spin
(the context's wait_limit_us).  tn_batch_debug_hold leaves one step's tiles out of the work list,
so its consumers wait for a producer that never runs -- a flag that nothing sets.  The wait must
give up, the job must report TN_ETIMEOUT, the launch-wide abort flag must end every other wait of
the launch at once, and the context must stay usable: the next run, with the full work list,
gives correct results on the same batch.
"""
import time

import numpy as np
import pytest

from oracle import statevector as sv
from paper_2507_20667_gb300 import inputs as tni
from parity import TOL, amplitude_bitstring, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnsa():
    from paper_2507_20667_gb300 import tnsa as mod
    return mod


def _batch(tnsa, limit_us, n_jobs=8):
    circ, _ = tni.cfg1()
    psi = sv.simulate(circ).reshape((2,) * 10)
    xs = [amplitude_bitstring(lambda y: psi[tuple(y)], 10, 500 + i, tni.random_bitstring)[0]
          for i in range(n_jobs)]
    refs = [psi[tuple(x)] for x in xs]
    hs = [tnsa.tn_build(tni.amplitude_tn(circ, x)) for x in xs]
    plan = tnsa.tn_plan_create(hs[0], k=1)
    ctx = tnsa.tn_ctx_create(0)
    tnsa.tn_ctx_set_config(ctx, local_budget=0, wait_limit_us=limit_us)   # every step global
    assert tnsa.tn_ctx_get_config(ctx)["wait_limit_us"] == limit_us
    b = tnsa.tn_batch_create(ctx, hs, [plan] * n_jobs, "c64")
    steps = tnsa.tn_plan_compile_steps(hs[0], plan, "c64", 0)
    return ctx, b, hs, refs, steps


def _run(tnsa, b, n):
    t0 = time.perf_counter()
    tnsa.tn_batch_run(b)
    mant, e2, st = tnsa.tn_batch_results(b, n)
    return mant * np.ldexp(1.0, e2), st, time.perf_counter() - t0


def test_held_dependency_times_out_and_context_recovers(tnsa):
    limit_us = 2000
    ctx, b, hs, refs, steps = _batch(tnsa, limit_us)
    n = len(hs)
    got, st, _ = _run(tnsa, b, n)                       # a normal run first
    assert (st == 0).all()
    tnsa.tn_batch_debug_hold(b, 3, 0)                   # step 0 of job 3 never runs
    got, st, secs = _run(tnsa, b, n)
    assert st[3] == tnsa.TN_ETIMEOUT
    assert set(st.tolist()) <= {0, tnsa.TN_ETIMEOUT}
    assert secs < 2.0, secs                              # one 2 ms time-out, not the default 4 s
    for i in np.flatnonzero(st == 0):                   # the jobs that were not held up are right
        check(got[i], refs[i], TOL["c64"], f"job {i} beside the held job")
    tnsa.tn_batch_debug_hold(b, -1, -1)                 # full work list again: same batch, same ctx
    got, st, _ = _run(tnsa, b, n)
    assert (st == 0).all()
    for i in range(n):
        check(got[i], refs[i], TOL["c64"], f"job {i} after recovery")
    # the context also still runs new work
    m, e, _ = tnsa.tn_contract(ctx, hs[0], tnsa.tn_plan_create(hs[0], k=1), "c64")
    check(tnsa.amplitude(m, e), refs[0], TOL["c64"], "tn_contract after recovery")


def test_abort_flag_ends_every_wait_of_the_launch(tnsa):
    """Every job held, with more waiting tiles (one per job) than the persistent kernel has
    resident blocks: the tiles claimed after the first wave of waits starts its waits only when a
    block frees up, about one wait limit in.  Without the abort flag those waits would run out on
    their own, doubling the launch; with it they give up at once, so the launch ends after about
    one limit, and every job reports TN_ETIMEOUT."""
    limit_us = 500000
    n_jobs = 2 * 152 * 2 + 16          # more than two resident blocks on each of the 152 SMs
    ctx, b, hs, refs, steps = _batch(tnsa, limit_us, n_jobs=n_jobs)
    n = len(hs)
    _run(tnsa, b, n)
    for j in range(n):
        tnsa.tn_batch_debug_hold(b, j, 0)
    got, st, secs = _run(tnsa, b, n)
    assert (st == tnsa.TN_ETIMEOUT).all()
    assert 0.9 * limit_us * 1e-6 <= secs < 1.5 * limit_us * 1e-6, secs
    tnsa.tn_batch_debug_hold(b, -1, -1)
    got, st, _ = _run(tnsa, b, n)
    assert (st == 0).all()
    for i in range(n):
        check(got[i], refs[i], TOL["c64"], f"job {i} after recovery")


def test_hold_rejects_bad_arguments(tnsa):
    ctx, b, hs, refs, steps = _batch(tnsa, 1000, n_jobs=2)
    with pytest.raises(tnsa.TnError):
        tnsa.tn_batch_debug_hold(b, 5, 0)
    with pytest.raises(tnsa.TnError):
        tnsa.tn_batch_debug_hold(b, 0, 10 ** 6)
    with pytest.raises(tnsa.TnError):
        tnsa.tn_ctx_set_config(ctx, wait_limit_us=0)
