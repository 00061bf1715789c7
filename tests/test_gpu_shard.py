"""The GPU form of interval sharding on one GPU: a process group of one rank (NCCL) whose
rank owns three consecutive interval ranges ("virtual" ranks), so the whole path runs --
partials by mg_set_controls / mg_evolve on each range, the NCCL all-gather, the ordered
combination by mg_cgemm on the device -- against the oracle and the unsharded evolution."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402
from paper_2411_09982_gb300 import shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("prec,tol", [(M.MG_PREC_SPLIT, 1e-6), (M.MG_PREC_FP64, 1e-11)])
def test_sharded_propagator_on_one_gpu_matches_oracle(prec, tol):
    import torch.distributed as dist
    wl = W.transmon_chain(n_sites=5, levels=3, J=0.01, seed=3, omega0_max=0.05, T=3.0, sigma=0.8, N=31, P=16,
                          unitary=True, name="chain243_U")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        ctx = M.Context(0)
        samples, w = M.node_samples(wl)
        S = torch.from_numpy(samples).cuda()
        H0, Hk = torch.from_numpy(wl.H0).cuda(), torch.from_numpy(wl.Hk).cuda()
        U = shard.evolve_propagator_sharded(ctx, H0, Hk, S, wl.N, wl.P, wl.t0, wl.dt, w, precision=prec,
                                            virtual=3)
        torch.cuda.synchronize()
        ref = oracle.evolve_workload(wl)
        err = np.abs(U.cpu().numpy() - ref).max()
        assert err <= tol, err
        whole, _ = M.evolve_workload(ctx, wl, prec, 6)
        assert np.abs(U.cpu().numpy() - whole.cpu().numpy()).max() <= tol
        ctx.close()
    finally:
        dist.destroy_process_group()
