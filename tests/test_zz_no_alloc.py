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


def _bound(A, B, d, L):
    # the tolerance of the split-product parity test (digit truncation + level->=3 rounding)
    beta = split_beta(d)
    ma = np.abs(np.stack([A.real, A.imag])).max()
    mb = np.abs(np.stack([B.real, B.imag])).max()
    return (L + 2) * 2 * d * (2 * ma) * (2 * mb) * (2.0 ** (-beta * L) + L * 2.0 ** (-22 - 3 * beta))


def test_static_scratch_product_matches_allocating_product_on_consecutive_calls():
    """Two calls in a row of the same size, then a larger call followed by a smaller one:
    nothing the larger call left in the shared scratch (digits, exponents, padding) may
    reach the smaller call's result."""
    ctx = M.Context(0)
    L = 6
    for call, (d, batch) in enumerate([(100, 3), (100, 3), (300, 2), (37, 4)]):
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
        bound = _bound(A, B, d, L)
        assert np.abs(got - want).max() <= bound, (call, d)
        assert np.abs(got - A @ B).max() <= bound, (call, d)
    ctx.close()


_FIRST_CALL = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from paper_2411_09982_gb300 import magnus as M
from tests.test_zz_no_alloc import _bound, rand_c
d, batch, L = 129, 2, 6
rng = np.random.default_rng(7)
A, B = rand_c(rng, (batch, d, d)), rand_c(rng, (batch, d, d))
Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
outs = [torch.full_like(Ad, float("nan")) for _ in range(3)]
s = torch.cuda.Stream()
torch.cuda.synchronize()
# the first library call of this process, on a torch stream, without any context
M.mg_cgemm_split_static(0, s, batch, d, Ad, Bd, outs[0], L)
free0 = torch.cuda.mem_get_info()[0]
for o in outs[1:]:
    M.mg_cgemm_split_static(0, s, batch, d, Ad, Bd, o, L)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
bound = _bound(A, B, d, L)
for o in outs:
    assert np.abs(o.cpu().numpy() - A @ B).max() <= bound
assert free1 == free0, (free0, free1)
print("FIRST_CALL_OK")
"""


def test_static_scratch_as_first_call_on_a_stream_allocates_nothing():
    """In a fresh process, the allocation-free product is the first library call (no
    context exists), runs on a non-default stream, matches A @ B, and repeated calls leave
    the device's free memory unchanged."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL.format(root=root)], capture_output=True, text=True,
                       timeout=300, cwd=root)
    assert r.returncode == 0 and "FIRST_CALL_OK" in r.stdout, r.stdout + r.stderr


def test_static_scratch_rejects_requests_beyond_its_size():
    d = 2048
    A = torch.zeros((1, d, d), dtype=torch.complex128, device="cuda")
    C = torch.empty_like(A)
    with pytest.raises(M.MagnusError) as e:
        M.mg_cgemm_split_static(0, None, 1, d, A, A, C, 6)
    assert e.value.code == M.MG_EUNSUPPORTED
