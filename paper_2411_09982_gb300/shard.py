"""Host-side logic for spreading Magnus work over several processes.

Two forms of parallelism exist on the path:

* independent jobs (instances, requests): replicas, no exchange;
* one job's N intervals cut into contiguous ranges, one per rank: every rank
  forms the partial product of its range, P_r = U_{end-1} ... U_{start}, and a
  single exchange (all-gather of the d x d partials) yields
  U(T) = P_{G-1} ... P_1 P_0 (later ranges on the left, as in the product of
  the first-order Magnus propagators).  For a state the exchange is lighter:
  psi passes along the ranks in time order, psi_{r+1} = P_r psi_r, one message
  of d complex values per hop, and the last rank broadcasts psi(T).

The exchange uses torch.distributed (NCCL between GPUs, gloo in the CPU tests).
Functions here hold no method arithmetic beyond that final ordered product of
the gathered partials.
"""
from __future__ import annotations

from typing import Callable, List, Tuple

import numpy as np


def interval_ranges(N: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous (start, count) per rank, counts differing by at most one."""
    if N < 1 or world < 1:
        raise ValueError("need N >= 1 and world >= 1")
    base, extra = divmod(N, world)
    out, start = [], 0
    for r in range(world):
        cnt = base + (1 if r < extra else 0)
        out.append((start, cnt))
        start += cnt
    return out


def combine_partials(partials) -> np.ndarray:
    """U = P_{G-1} ... P_0 for partials listed in rank (= time) order; empty ranges are identities."""
    acc = None
    for P in partials:
        if P is None:
            continue
        acc = P.copy() if acc is None else P @ acc
    return acc


def sharded_propagator(local_partial: Callable[[int, int], np.ndarray], N: int, d: int, group=None) -> np.ndarray:
    """Every rank calls this with the same N, d: it computes its own range's partial product
    with `local_partial(start, count)` (identity for an empty range), all-gathers the partials
    and returns the full propagator on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    start, count = interval_ranges(N, world)[rank]
    P = local_partial(start, count) if count > 0 else np.eye(d, dtype=np.complex128)
    t = torch.from_numpy(np.ascontiguousarray(P)).view(torch.float64)
    gathered = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(gathered, t, group=group)
    parts = [g.view(torch.complex128).numpy() for g in gathered]
    return combine_partials(parts)


def sharded_state(local_partial: Callable[[int, int], np.ndarray], N: int, d: int, psi0, group=None) -> np.ndarray:
    """State form of the interval sharding.  Every rank calls this with the same N, d and
    psi0: it forms its own range's partial product with `local_partial(start, count)` (all
    ranks at once), then the state passes from rank to rank in time order (rank r receives
    psi_r, applies P_r, sends psi_{r+1}; a rank with an empty range passes psi on), and the
    last rank broadcasts psi(T), which every rank returns."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)

    def glob(r):
        return r if group is None else dist.get_global_rank(group, r)

    start, count = interval_ranges(N, world)[rank]
    P = local_partial(start, count) if count > 0 else None
    buf = torch.empty(2 * d, dtype=torch.float64)
    if rank == 0:
        psi = np.asarray(psi0, dtype=np.complex128).copy()
    else:
        dist.recv(buf, src=glob(rank - 1), group=group)
        psi = buf.view(torch.complex128).numpy().copy()
    if P is not None:
        psi = P @ psi
    if rank < world - 1:
        dist.send(torch.from_numpy(np.ascontiguousarray(psi)).view(torch.float64), dst=glob(rank + 1), group=group)
    else:
        buf.copy_(torch.from_numpy(np.ascontiguousarray(psi)).view(torch.float64))
    dist.broadcast(buf, src=glob(world - 1), group=group)
    return buf.view(torch.complex128).numpy().copy()


def max_over_ranks(value: float, group=None) -> float:
    """The slowest rank's time (what a multi-GPU step costs)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
