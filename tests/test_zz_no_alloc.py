"""The allocation-free product (mg_cgemm_split_static) against mg_cgemm.

mg_cgemm_split_static serves callers that cannot allocate device memory: its
scratch is a static device array inside the library instead of cudaMalloc.  It
must return what the allocating entry point returns for the same inputs, on
every call, although all calls reuse the same scratch.  This file is collected
after the parity tests, so that a failure here leaves them already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


def split_beta(d):
    for beta in range(8, 1, -1):
        if 2.0 ** (2 * beta - 1) * 2 * d <= 2.0 ** 24:
            return beta
    return 2


def rand_c(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_static_scratch_product_matches_allocating_product_on_consecutive_calls():
    ctx = M.Context(0)
    d, batch, L = 100, 3, 6
    for call in range(2):
        rng = np.random.default_rng(1000 + call)
        A, B = rand_c(rng, (batch, d, d)), rand_c(rng, (batch, d, d))
        Ad = torch.from_numpy(A).cuda()
        Bd = torch.from_numpy(B).cuda()
        ref = torch.empty_like(Ad)
        M.mg_cgemm(ctx, batch, d, Ad, Bd, ref, M.MG_PREC_SPLIT, L)
        out = torch.full_like(Ad, float("nan"))
        M.mg_cgemm_split_static(0, None, batch, d, Ad, Bd, out, L)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        # same tolerance as the split-product parity test (digit truncation + level->=3 rounding)
        beta = split_beta(d)
        ma = np.abs(np.stack([A.real, A.imag])).max()
        mb = np.abs(np.stack([B.real, B.imag])).max()
        bound = (L + 2) * 2 * d * (2 * ma) * (2 * mb) * (2.0 ** (-beta * L) + L * 2.0 ** (-22 - 3 * beta))
        assert np.abs(got - want).max() <= bound
        assert np.abs(got - A @ B).max() <= bound
    ctx.close()


def test_static_scratch_rejects_requests_beyond_its_size():
    d = 2048
    A = torch.zeros((1, d, d), dtype=torch.complex128, device="cuda")
    C = torch.empty_like(A)
    with pytest.raises(M.MagnusError) as e:
        M.mg_cgemm_split_static(0, None, 1, d, A, A, C, 6)
    assert e.value.code == M.MG_EUNSUPPORTED
