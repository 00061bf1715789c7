"""Resuming an evolution at an interval boundary, chunk boundaries, and evolutions
without the trace shift.

* Resume: a first mg_evolve over intervals 0..n-1 returns psi_n (or U_{n-1} ... U_0);
  a second call with controls for the remaining intervals (t0 moved to t0 + n dt)
  takes it as its input.  Together they must give the oracle's single evolution:
  the state continues from psi_n, and the propagator output is U(T) U0 with U0 the
  first part.
* Chunks: a context whose workspace limit is 1 MiB processes a few intervals per
  chunk, so the running product, the state and the re-orthonormalisation period
  cross many chunk boundaries.
* MG_FLAG_NO_TRACE_SHIFT: the exponent keeps its trace, and the phase is carried by
  the polynomial and the squarings instead of an exact factor.

This file is collected late in the GPU suite, just before the allocation-free product's.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    M.load()
    c = M.Context(0)
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("prec,L,tol", [(M.MG_PREC_FP64, 6, 1e-11), (M.MG_PREC_SPLIT, 6, 1e-6)])
def test_two_calls_resumed_at_an_interval_equal_one_evolution(ctx, prec, L, tol):
    n = 23
    for wl in (W.config(0, N=60), W.transmon_resonator(nt=3, nr=10, N=60, unitary=True)):
        state = wl.psi0 is not None
        kind = M.MG_OUT_STATE if state else M.MG_OUT_PROPAGATOR
        shape = (wl.d,) if state else (wl.d, wl.d)
        samples, w = M.node_samples(wl)
        plan = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), prec, L)
        try:
            mid = torch.empty(shape, dtype=torch.complex128, device="cuda")
            out = torch.empty(shape, dtype=torch.complex128, device="cuda")
            plan.set_controls(n, wl.P, wl.t0, wl.dt, w, cuda(samples[:n]))
            plan.evolve(kind, cuda(wl.psi0) if state else None, mid, report=False)
            plan.set_controls(wl.N - n, wl.P, wl.t0 + n * wl.dt, wl.dt, w, cuda(samples[n:]))
            plan.evolve(kind, mid, out, report=False)
            torch.cuda.synchronize()
        finally:
            plan.close()
        ref = oracle.evolve_workload(wl)
        err = np.abs(out.cpu().numpy() - ref).max()
        assert err <= tol, (wl.name, err)


@pytest.fixture(scope="module")
def small_ctx():
    M.load()
    c = M.Context(0, workspace_limit=1 << 20)
    yield c
    c.close()


@pytest.mark.parametrize("prec,L,tol", [(M.MG_PREC_FP64, 6, 1e-11), (M.MG_PREC_SPLIT, 6, 1e-6)])
@pytest.mark.parametrize("reorth", [0, 7])
def test_evolutions_across_many_chunks(small_ctx, prec, L, tol, reorth):
    for wl in (W.config(0, N=100), W.transmon_resonator(nt=3, nr=10, N=60, unitary=True)):
        out, _ = M.evolve_workload(small_ctx, wl, prec, L, reorth_every=reorth)
        err = np.abs(out.cpu().numpy() - oracle.evolve_workload(wl)).max()
        assert err <= tol, (wl.name, err)


def test_evolution_without_the_trace_shift(ctx):
    """FP64 without the shift: the exponent's 1-norm roughly doubles (the trace part is
    ~57 rad per interval here), so the rounding scale u ||Hbar||_1 N grows with it."""
    for wl in (W.config(0, N=100), W.transmon_resonator(nt=3, nr=10, N=60, unitary=True)):
        out, rep = M.evolve_workload(ctx, wl, M.MG_PREC_FP64, flags=M.MG_FLAG_NO_TRACE_SHIFT)
        err = np.abs(out.cpu().numpy() - oracle.evolve_workload(wl)).max()
        assert err <= 1e-10, (wl.name, err)
