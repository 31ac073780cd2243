"""GPU permutation kernel (the transposition of TTGT) against numpy.transpose on an iota payload:
index maps must agree bit for bit."""
import numpy as np
import pytest

from oracle import perm as operm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2507_20667_gb300 import tnsa
    ctx = tnsa.tn_ctx_create(0, stream=torch.cuda.current_stream().cuda_stream)
    return torch, tnsa, ctx


CASES = [
    ((2,) * 10, None), ((2,) * 20, None), ((3, 5, 7, 2), None), ((33, 65, 3), None),
    ((1, 7, 1, 9), None), ((1000, 1000), (1, 0)), ((4, 4, 4, 4, 4, 4), None), ((17,), (0,)),
    ((2,) * 24, None), ((6, 1, 8, 31, 2), None),
    # the innermost axis survives: rows copied whole (16-byte vectors when aligned, and short rows)
    ((8, 16, 64), (1, 0, 2)), ((2,) * 12, (3, 1, 0, 2, 4, 5, 6, 7, 8, 9, 10, 11)), ((5, 7, 3), (1, 0, 2)),
    ((4, 6, 10), (1, 0, 2)), ((3, 3, 5), (0, 1, 2)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("elem", [4, 8, 16])
def test_permute_iota_bit_exact(env, case, elem):
    torch, tnsa, ctx = env
    dims, perm = CASES[case]
    rng = np.random.default_rng(case * 10 + elem)
    if perm is None:
        perm = tuple(int(p) for p in rng.permutation(len(dims)))
    n = int(np.prod(dims))
    want = operm.permute_iota(dims, perm, dtype=np.uint32)
    # payload: element i holds iota value i in its first 4 bytes, a fingerprint in the rest
    words = elem // 4
    src = np.zeros((n, words), np.int32)
    src[:, 0] = np.arange(n, dtype=np.int64).astype(np.int32)
    for w in range(1, words):
        src[:, w] = (np.arange(n, dtype=np.int64) * (w + 7) + 3).astype(np.int32)
    d_in = torch.from_numpy(src).cuda()
    d_out = torch.full_like(d_in, -1)
    tnsa.tn_permute(ctx, d_in.data_ptr(), d_out.data_ptr(), elem, dims, perm)
    torch.cuda.synchronize()
    out = d_out.cpu().numpy()
    assert np.array_equal(out[:, 0].astype(np.uint32), want)
    for w in range(1, words):
        assert np.array_equal(out[:, w], src[want.astype(np.int64), w])


def test_permute_rejects_bad_perm(env):
    torch, tnsa, ctx = env
    x = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(tnsa.TnError):
        tnsa.tn_permute(ctx, x.data_ptr(), x.data_ptr(), 8, (2, 4), (0, 0))
