"""Sliced contraction on the GPU (Section 4.1): the slices run as the jobs of a batch and their
values are summed in FP64; the sum equals the unsliced contraction and the state vector."""
import pytest

from oracle import statevector as sv
from paper_2507_20667_gb300 import inputs as tni
from parity import TOL, amplitude_bitstring, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnsa():
    from paper_2507_20667_gb300 import tnsa as mod
    return mod


@pytest.mark.parametrize("prec", ["c128", "c64", "bf16"])
def test_sliced_equals_unsliced_and_state_vector(tnsa, prec):
    circ, _ = tni.cfg3(small=True)
    x, ref, _ = amplitude_bitstring(lambda y: sv.amplitude(circ, y), 20, 1003, tni.random_bitstring)
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=8, iterations=100, seed=7, position=net.qubit)
    mem = tnsa.tn_plan_counts(plan)[2]
    r = tnsa.tn_plan_slice(h, plan, mem // 64)
    assert r["n_slices"] >= 16
    ctx = tnsa.tn_ctx_create(0)
    m, e, ns = tnsa.tn_contract_sliced(ctx, h, plan, r["edges"], prec, max_jobs=37)   # ragged last batch
    assert ns == r["n_slices"]
    check(complex(m) * 2.0 ** e, ref, TOL[prec], "sliced")
    m0, e0, _ = tnsa.tn_contract(ctx, h, plan, prec)
    check(tnsa.amplitude(m0, e0), ref, TOL[prec], "unsliced")
