"""A batch captured once in a CUDA graph (mg_batch_graph_*) against the CPU oracle.

The captured batch takes each interval's own squaring count on the device and issues
no host synchronisation between its launches; a replay evolves whatever the plans'
coefficient buffers and the input buffers hold at launch time.  Tolerances: the stated
1e-6 (split) and the FP64 bound of test_gpu_parity (1e-11, or 4 u |Hbar|_1 N on the
random jobs with very long intervals)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def scaled_drive(wl, f):
    """The same job with every control signal scaled by f (new samples, same shape)."""
    import dataclasses
    base = wl.drive
    return dataclasses.replace(wl, drive=lambda t: f * base(t))


def ref_and_tol(wl, prec):
    ref, parts = oracle.evolve_workload(wl, return_parts=True)
    if prec == M.MG_PREC_SPLIT:
        return ref, 1e-6
    hmax = max(np.abs(h).sum(axis=0).max() for h in parts["Hbar"])
    return ref, max(1e-11, 4 * 2.0 ** -53 * hmax * wl.N)


def jobs_mix(seed=41, n=9):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        wl = W.random_instance(rng, name=f"g{i}", N_range=(5, 60), d_range=(16, 140))
        if i % 3 == 1:
            wl.psi0 = None
        jobs.append(wl)
    jobs.append(W.transmon_resonator(nt=3, nr=10, N=70, name="d30"))
    jobs.append(W.transmon_chain(n_sites=5, levels=3, J=0.01, seed=2, omega0_max=0.05, T=2.0, sigma=0.5, N=9,
                                 P=16, unitary=True, name="chain243"))
    return jobs


def make(ctx, jobs, prec):
    plans, kinds, ins, outs = [], [], [], []
    for wl in jobs:
        samples, w = M.node_samples(wl)
        p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), prec, 6)
        p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
        plans.append(p)
        state = wl.psi0 is not None
        kinds.append(M.MG_OUT_STATE if state else M.MG_OUT_PROPAGATOR)
        ins.append(cuda(wl.psi0) if state else None)
        outs.append(torch.empty(wl.d if state else (wl.d, wl.d), dtype=torch.complex128, device="cuda"))
    return plans, kinds, ins, outs


@pytest.mark.parametrize("prec", [M.MG_PREC_SPLIT, M.MG_PREC_FP64])
def test_captured_batch_matches_oracle_on_replays(prec):
    stream = torch.cuda.Stream()
    ctx = M.Context(0, stream)
    jobs = jobs_mix()
    plans, kinds, ins, outs = make(ctx, jobs, prec)
    g = M.BatchGraph(ctx, plans, kinds, ins, outs)
    try:
        st = g.stats()
        assert st["kernel_nodes"] > 0 and st["nodes"] >= st["kernel_nodes"]
        for rep in range(2):
            for o in outs:
                o.fill_(float("nan"))
            torch.cuda.synchronize()
            assert g.launch() == [0] * len(jobs)
            for wl, o in zip(jobs, outs):
                ref, tol = ref_and_tol(wl, prec)
                err = np.abs(o.cpu().numpy() - ref).max()
                assert err <= tol, (rep, wl.name, wl.d, wl.N, err, tol)
        # new drive samples of the same shape: the replay evolves them
        for p, wl in zip(plans, jobs):
            wl2 = scaled_drive(wl, 0.5)
            samples, w = M.node_samples(wl2)
            p.set_controls(wl2.N, wl2.P, wl2.t0, wl2.dt, w, cuda(samples))
        assert g.launch() == [0] * len(jobs)
        for wl, o in zip(jobs, outs):
            ref, tol = ref_and_tol(scaled_drive(wl, 0.5), prec)
            assert np.abs(o.cpu().numpy() - ref).max() <= tol, wl.name
        # a plan whose interval count changed cannot replay the capture
        samples, w = M.node_samples(jobs[0], jobs[0].N + 1)
        plans[0].set_controls(jobs[0].N + 1, jobs[0].P, jobs[0].t0, jobs[0].dt, w, cuda(samples))
        with pytest.raises(M.MagnusError) as e:
            g.launch()
        assert e.value.code == M.MG_EINVAL
    finally:
        g.close()
        for p in plans:
            p.close()
        ctx.close()


def test_captured_batch_nonfinite_job_fails_alone_and_legacy_stream_rejected():
    stream = torch.cuda.Stream()
    ctx = M.Context(0, stream)
    jobs = jobs_mix(seed=43, n=5)
    plans, kinds, ins, outs = make(ctx, jobs, M.MG_PREC_SPLIT)
    g = M.BatchGraph(ctx, plans, kinds, ins, outs)
    try:
        samples, w = M.node_samples(jobs[2])
        samples = samples.copy()
        samples[1, 2, 0] = np.nan
        plans[2].set_controls(jobs[2].N, jobs[2].P, jobs[2].t0, jobs[2].dt, w, cuda(samples))
        status = g.launch()
        assert status[2] == M.MG_ENONFINITE
        for i, (wl, o) in enumerate(zip(jobs, outs)):
            if i == 2:
                continue
            assert status[i] == 0
            ref, tol = ref_and_tol(wl, M.MG_PREC_SPLIT)
            assert np.abs(o.cpu().numpy() - ref).max() <= tol
    finally:
        g.close()
        for p in plans:
            p.close()
        ctx.close()
    ctx0 = M.Context(0)   # legacy default stream
    p = M.Plan(ctx0, cuda(jobs[0].H0), cuda(jobs[0].Hk), M.MG_PREC_SPLIT, 6)
    samples, w = M.node_samples(jobs[0])
    p.set_controls(jobs[0].N, jobs[0].P, jobs[0].t0, jobs[0].dt, w, cuda(samples))
    o = torch.empty((jobs[0].d,), dtype=torch.complex128, device="cuda")
    with pytest.raises(M.MagnusError) as e:
        M.BatchGraph(ctx0, [p], [M.MG_OUT_STATE], [cuda(jobs[0].psi0)], [o])
    assert e.value.code == M.MG_EINVAL
    p.close()
    ctx0.close()
