"""Gloo tests (CPU, world size 2 and 3) of the multi-process path: interval-range sharding of
one job with a single all-gather of partial products, the state form that passes psi from
rank to rank, and the max-over-ranks timing reduction.  The partial products come from the
CPU oracle and the products of the exchange from a torch CPU stand-in (on GPUs they are the
library's mg_evolve and mg_cgemm; see test_gpu_shard.py)."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2411_09982_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q, virtual=1):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.transmon_resonator(nt=3, nr=4, N=37, T=3.0, sigma=0.7, omega0=0.4, unitary=True)
        x, w = oracle.gauss_legendre(wl.P)

        def local_partial(start, count):
            t = oracle.node_times(wl.t0 + start * wl.dt, wl.dt, count, x)
            U, _, _ = oracle.interval_propagators(wl.H0, wl.Hk, wl.drive(t), w, wl.dt)
            return torch.from_numpy(oracle.propagate_unitary(U))

        U = shard.sharded_propagator(local_partial, wl.N, wl.d, lambda A, B: A @ B, virtual=virtual)
        slowest = shard.max_over_ranks(1.0 + rank)
        q.put((rank, U.numpy(), slowest))
    finally:
        dist.destroy_process_group()


def test_interval_ranges_cover_in_order():
    for N in (1, 2, 7, 100):
        for world in (1, 2, 3, 8):
            r = shard.interval_ranges(N, world)
            assert sum(c for _, c in r) == N
            assert all(r[i][0] + r[i][1] == r[i + 1][0] for i in range(len(r) - 1))
            assert max(c for _, c in r) - min(c for _, c in r) <= 1


def test_combine_partials_orders_later_on_the_left():
    import torch
    rng = np.random.default_rng(0)
    P = [torch.from_numpy(rng.normal(size=(3, 3))) for _ in range(3)]
    got = shard.combine_partials([P[0], None, P[1], P[2]], lambda A, B: A @ B)
    np.testing.assert_allclose(got.numpy(), (P[2] @ P[1] @ P[0]).numpy())


@pytest.mark.timeout(180)
@pytest.mark.parametrize("virtual", [1, 3])
def test_two_rank_sharded_propagator_matches_single_process(virtual):
    """Two ranks, each owning one range (or three consecutive ranges): one all-gather and
    the ordered product give the single-process propagator on every rank."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, virtual)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=150) for _ in range(2)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    wl = W.transmon_resonator(nt=3, nr=4, N=37, T=3.0, sigma=0.7, omega0=0.4, unitary=True)
    ref = oracle.evolve_workload(wl)
    for rank, U, slowest in results:
        np.testing.assert_allclose(U, ref, atol=1e-12, rtol=0)
        assert slowest == 2.0


def _state_worker(rank, world, port, N, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.transmon_resonator(nt=3, nr=4, N=N, T=3.0, sigma=0.7, omega0=0.4)
        x, w = oracle.gauss_legendre(wl.P)

        def local_partial(start, count):
            t = oracle.node_times(wl.t0 + start * wl.dt, wl.dt, count, x)
            U, _, _ = oracle.interval_propagators(wl.H0, wl.Hk, wl.drive(t), w, wl.dt)
            return torch.from_numpy(oracle.propagate_unitary(U))

        psi = shard.sharded_state(local_partial, wl.N, wl.d, torch.from_numpy(wl.psi0), lambda P, v: P @ v)
        q.put((rank, psi.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("world,N", [(2, 37), (3, 37), (3, 2)])
def test_sharded_state_matches_single_process(world, N):
    """psi(T) from ranks that each own a range of intervals (N = 2 over 3 ranks leaves one
    range empty) equals the single-process evolution on every rank."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_state_worker, args=(r, world, port, N, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=150) for _ in range(world)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    wl = W.transmon_resonator(nt=3, nr=4, N=N, T=3.0, sigma=0.7, omega0=0.4)
    assert wl.psi0 is not None
    ref = oracle.evolve_workload(wl)
    assert sorted(r for r, _ in results) == list(range(world))
    for _, psi in results:
        np.testing.assert_allclose(psi, ref, atol=1e-12, rtol=0)


def _failing_worker(rank, world, port, q):
    import datetime
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    d = 4

    def local_partial(start, count):
        if rank == 1:
            raise RuntimeError("rank 1 failed while forming its partial product")
        return torch.eye(d, dtype=torch.complex128)

    try:
        shard.sharded_state(local_partial, 8, d, torch.eye(d, dtype=torch.complex128)[0], lambda P, v: P @ v)
        q.put((rank, "ok"))
    except Exception as e:   # the failure reaches every rank as an exception, not a hang
        q.put((rank, type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


@pytest.mark.timeout(120)
def test_rank_failure_surfaces_as_an_error_on_the_other_rank():
    """A rank that fails before its exchange: the rank waiting for its message gets an error
    from the process group (peer gone or timeout) instead of waiting forever."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=90) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
    assert results[1] == "RuntimeError"
    assert results[0] != "ok", results
