"""The allocation-free inner product (tn_dot_noalloc) against numpy and the existing entry point.

tn_dot_noalloc serves callers that must not allocate device memory while they run (their device
memory belongs to a host framework's pool, or a serving loop cannot afford cudaMalloc's implicit
synchronization or its failure mid-request).  Its scratch is a fixed device array shared by all
calls, so this test calls it twice in a row on the same array and compares both results with
numpy (complex128 products of the vectors as stored on the device, so independent of every GPU
path) and with tn_contract on the same two vectors written as a two-tensor network (one shared
leg).  This file is collected last, so a run that stops at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-12}


class _TwoVectors:
    def __init__(self, a, b):
        self.degrees = np.array([1, 1], np.int32)
        self.dims = np.array([len(a), len(b)], np.int64)
        self.data = np.concatenate([a, b]).astype(np.complex128).view(np.float64)
        self.edges = np.array([[0, 0, 1, 0]], np.int32)


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_dot_noalloc_matches_contract(prec):
    import torch
    from paper_2507_20667_gb300 import tnsa
    rng = np.random.default_rng(11)
    n = 3 * 65536 + 12345                       # several scratch slots and a ragged tail
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2)
    b = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2)
    net = tnsa.tn_build(_TwoVectors(a, b))
    plan = tnsa.tn_plan_create(net, k=1)
    ctx = tnsa.tn_ctx_create(0)
    m, e, _ = tnsa.tn_contract(ctx, net, plan, prec)
    ref = complex(m) * 2.0 ** e
    dt = torch.complex64 if prec == "c64" else torch.complex128
    d_a = torch.from_numpy(a).to(dt).cuda()
    d_b = torch.from_numpy(b).to(dt).cuda()
    # numpy: the vectors as the device holds them, multiplied and summed in complex128
    exact = complex(np.dot(d_a.cpu().numpy().astype(np.complex128), d_b.cpu().numpy().astype(np.complex128)))
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        tnsa.tn_dot_noalloc(0, stream, d_a.data_ptr(), d_b.data_ptr(), n, prec, out.data_ptr())
        torch.cuda.synchronize()
        assert torch.cuda.current_device() == 0        # the caller's current device is kept
        got = complex(out[0].item(), out[1].item())
        assert abs(got - exact) <= TOL[prec] * abs(exact), (call, got, exact)
        assert abs(got - ref) <= TOL[prec] * abs(ref), (call, got, ref)


def test_dot_noalloc_rejects_oversize():
    import torch
    from paper_2507_20667_gb300 import tnsa
    buf = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(tnsa.TnError) as ei:
        tnsa.tn_dot_noalloc(0, 0, buf.data_ptr(), buf.data_ptr(), 2 ** 26 + 1, "c64", out.data_ptr())
    assert ei.value.status == tnsa.TN_EINVAL


def test_dot_noalloc_empty_vector():
    import torch
    from paper_2507_20667_gb300 import tnsa
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    tnsa.tn_dot_noalloc(0, 0, 0, 0, 0, "c64", out.data_ptr())
    torch.cuda.synchronize()
    assert out.tolist() == [0.0, 0.0]
