"""Failure detection of the tensor-core product without a GPU fault.

Every mbarrier wait of the split product's kernel is bounded.  The context's stall
test makes the MMA issuer of every CTA wait on a barrier that nothing completes: with
a 2 ms limit each CTA gives up, records the timeout and winds down (the loader still
waits for its own copies, the accumulator wait keeps its long limit), and the call
returns MG_ETIMEOUT.  The same context then computes a normal product.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


def rand_c(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("cta_pairs", [False, True])
def test_bounded_wait_runs_out_and_context_recovers(cta_pairs):
    """With cta_pairs the product of d = 200 runs on 2-CTA clusters: rank 0's MMA issuer
    gives up, hands its verdict to both CTAs, and both wind down through the closing
    cluster barrier."""
    ctx = M.Context(0)
    ctx.set_cta_pairs(cta_pairs)
    try:
        rng = np.random.default_rng(3)
        d, batch = 200, 2
        A, B = rand_c(rng, (batch, d, d)), rand_c(rng, (batch, d, d))
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        C = torch.zeros_like(Ad)
        ctx.set_wait_limit(0.002, stall_test=True)
        with pytest.raises(M.MagnusError) as e:
            M.mg_cgemm(ctx, batch, d, Ad, Bd, C, M.MG_PREC_SPLIT, 6)
        assert e.value.code == M.MG_ETIMEOUT
        # the limit alone (no stall) does not fail a product whose operands arrive
        ctx.set_wait_limit(0.5, stall_test=False)
        M.mg_cgemm(ctx, batch, d, Ad, Bd, C, M.MG_PREC_SPLIT, 6)
        ctx.set_wait_limit(4.0, stall_test=False)
        M.mg_cgemm(ctx, batch, d, Ad, Bd, C, M.MG_PREC_SPLIT, 6)
        torch.cuda.synchronize()
        assert np.abs(C.cpu().numpy() - A @ B).max() <= 1e-9 * np.abs(A @ B).max()
        with pytest.raises(M.MagnusError):
            ctx.set_wait_limit(5.0)
    finally:
        ctx.close()
