"""The autotuner on the GPU: the configuration it measures and sets meets the oracle within
the requested tolerance, a second tuning of the same job comes from the cache, and a
server takes a tuned configuration for a job submitted with MG_PREC_AUTO."""
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


CASES = [
    # (workload, tolerance)
    (W.config(0, N=300), 1e-6),                                   # d = 30 state
    (W.config(0, N=300), 1e-11),                                  # the same, FP64-level tolerance
    (W.transmon_chain(n_sites=4, levels=3, J=0.01, seed=3, omega0_max=0.05, T=10.0, sigma=2.0, N=200, P=16,
                      unitary=True, name="chain81_U"), 1e-7),     # d = 81 propagator
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tuned_configuration_meets_the_tolerance(case, tmp_path):
    wl, tol = CASES[case]
    cache = str(tmp_path / "tune.txt")
    ctx = M.Context(0)
    samples, w = M.node_samples(wl)
    plan = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_SPLIT, 6)
    plan.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
    output = M.MG_OUT_STATE if wl.psi0 is not None else M.MG_OUT_PROPAGATOR
    t0 = time.perf_counter()
    chosen = plan.autotune(output, tol, cache)
    t_first = time.perf_counter() - t0
    assert chosen["error"] * 4 <= tol and chosen["us_per_interval"] > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    if output == M.MG_OUT_STATE:
        out = torch.empty(wl.d, dtype=torch.complex128, device="cuda")
        plan.evolve(output, cuda(wl.psi0), out)
    else:
        out = torch.empty((wl.d, wl.d), dtype=torch.complex128, device="cuda")
        plan.evolve(output, None, out)
    torch.cuda.synchronize()
    err = np.abs(out.cpu().numpy() - oracle.evolve_workload(wl)).max()
    assert err <= tol, (wl.name, tol, chosen, err)
    # the second tuning of the same job is a cache hit: same choice, nothing measured
    t0 = time.perf_counter()
    again = plan.autotune(output, tol, cache)
    assert again == chosen and time.perf_counter() - t0 < max(0.5, 0.5 * t_first)
    assert len(open(cache).read().splitlines()) == 1
    plan.close()
    ctx.close()
    print(f"{wl.name} tol {tol:g}: {chosen}, error {err:.2e}")


def test_server_takes_the_tuned_configuration(tmp_path):
    cache = str(tmp_path / "tune.txt")
    wl = W.transmon_resonator(nt=3, nr=8, N=120, name="tr24")
    ctx = M.Context(0)
    samples, w = M.node_samples(wl)
    plan = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_SPLIT, 6)
    plan.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
    chosen = plan.autotune(M.MG_OUT_STATE, 1e-9, cache)
    plan.close()
    ctx.set_tune_cache(cache)
    srv = M.Server(ctx, mem_budget_bytes=1 << 30, quantum_intervals=32)
    out = torch.empty(wl.d, dtype=torch.complex128, device="cuda")
    keep = (cuda(wl.H0), cuda(wl.Hk), cuda(samples), cuda(wl.psi0))
    jid = srv.submit(keep[0], keep[1], wl.N, wl.P, wl.t0, wl.dt, w, keep[2], M.MG_OUT_STATE, keep[3], out,
                     precision=M.MG_PREC_AUTO, slices=0, tolerance=1e-9)
    assert jid is not None
    assert srv.wait(jid, 60.0)["status"] == 0
    torch.cuda.synchronize()
    err = np.abs(out.cpu().numpy() - oracle.evolve_workload(wl)).max()
    assert err <= 1e-9, (chosen, err)
    srv.close()
    ctx.close()
