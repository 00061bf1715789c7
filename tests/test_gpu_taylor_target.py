"""The Taylor truncation target (mg_plan_set_taylor_target) on the GPU.

It changes only the exponential's degree and squaring count (App. A.5's scaling and
squaring): a coarser target takes fewer squarings, every result stays within the split
tolerance of the oracle, and a plan batched alone agrees bit for bit with the same plan
in a batch of plans with other targets (the batch groups plans by target).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _plan(ctx, wl, u):
    sn, w = M.node_samples(wl)
    p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_SPLIT, 6)
    p.set_taylor_target(u)
    p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(sn))
    return p


def test_targets_alone_and_batched_agree_and_meet_the_tolerance():
    wl = W.transmon_chain(n_sites=4, levels=3, J=0.01, seed=5, omega0_max=0.05, T=20.0, sigma=4.0, N=150, P=16,
                          unitary=False, name="chain81_state")
    ref = oracle.evolve_workload(wl)
    # ||Hbar_n - tau_n I||_1 = 16.6 for every interval: 4 squarings at the digits' own
    # roundoff, 3 at both coarser targets (degree 18 throughout; an emulation of that
    # polynomial in FP64 errs by 9.8e-9 with 3 squarings)
    targets = [0.0, 2.0 ** -34, 2.0 ** -30]
    ctx = M.Context(0)
    alone, squarings = [], []
    for u in targets:
        p = _plan(ctx, wl, u)
        out = torch.empty(wl.d, dtype=torch.complex128, device="cuda")
        rep = p.evolve(M.MG_OUT_STATE, cuda(wl.psi0), out)
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
        squarings.append(rep["max_squarings"])
        p.close()
        assert np.abs(alone[-1] - ref).max() <= 1e-6, (u, np.abs(alone[-1] - ref).max())
    assert squarings == [4, 3, 3], squarings
    batched_alone = []
    for u in targets:
        p = _plan(ctx, wl, u)
        o = torch.empty(wl.d, dtype=torch.complex128, device="cuda")
        assert list(M.mg_evolve_batch(ctx, [p], [M.MG_OUT_STATE], [cuda(wl.psi0)], [o])) == [0]
        torch.cuda.synchronize()
        batched_alone.append(o.cpu().numpy())
        p.close()
        assert np.abs(batched_alone[-1] - ref).max() <= 1e-6
    plans = [_plan(ctx, wl, u) for u in targets]
    outs = [torch.empty(wl.d, dtype=torch.complex128, device="cuda") for _ in targets]
    status = M.mg_evolve_batch(ctx, plans, [M.MG_OUT_STATE] * len(targets), [cuda(wl.psi0)] * len(targets), outs)
    torch.cuda.synchronize()
    assert list(status) == [0] * len(targets)
    for o, a in zip(outs, batched_alone):
        assert np.array_equal(o.cpu().numpy(), a)
    for p in plans:
        p.close()
    ctx.close()


def test_target_outside_its_range_is_rejected():
    wl = W.config(0, N=10)
    ctx = M.Context(0)
    p = _plan(ctx, wl, 0.0)
    for bad in (-1e-12, 2e-3, float("nan")):
        with pytest.raises(M.MagnusError) as e:
            p.set_taylor_target(bad)
        assert e.value.code == M.MG_EINVAL
    p.close()
    ctx.close()
