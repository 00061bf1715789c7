"""Spreading one Magnus job over several processes (one GPU each).

Two forms of parallelism exist on the path:

* independent jobs (instances, requests): replicas, no exchange;
* one job's N intervals cut into contiguous ranges, one per rank: every rank
  forms the partial product of its range, P_r = U_{end-1} ... U_{start}, and a
  single exchange (all-gather of the d x d partials) yields
  U(T) = P_{G-1} ... P_1 P_0 (later ranges on the left, as in the product of
  the first-order Magnus propagators).  For a state the exchange is lighter:
  psi passes along the ranks in time order, psi_{r+1} = P_r psi_r, one message
  of d complex values per hop, and the last rank broadcasts psi(T).

The exchange uses torch.distributed on whatever tensors the caller hands over
(device tensors over NCCL between GPUs, CPU tensors over gloo).  Nothing here
multiplies: the partial products, the ordered combination and the application
to a state are the caller's functions -- on GPUs the library's own calls
(`evolve_propagator_sharded`: mg_evolve for the partials, mg_cgemm for the
combination).  Each rank may also own several consecutive ranges ("virtual"
ranks), which lets one GPU exercise the whole exchange-and-combine path.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple


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


def combine_partials(partials, mul: Callable):
    """U = P_{G-1} ... P_0 for partials listed in time order (None: an empty range),
    with the caller's product mul(A, B) = A B."""
    acc = None
    for P in partials:
        if P is None:
            continue
        acc = P.clone() if acc is None else mul(P, acc)
    return acc


def sharded_propagator(local_partial: Callable, N: int, d: int, mul: Callable, group=None, virtual: int = 1,
                       device=None):
    """Every rank calls this with the same N and d.  The N intervals are cut into
    world * virtual ranges; rank r owns ranges r*virtual .. r*virtual + virtual - 1 and forms
    each one's partial product with local_partial(start, count) (a complex128 tensor; not
    called for an empty range, which counts as the identity).  One all-gather exchanges the
    partials; every rank returns U(T) = P_last ... P_0 formed with mul."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    ranges = interval_ranges(N, world * virtual)
    mine = []
    for v in range(virtual):
        start, count = ranges[rank * virtual + v]
        mine.append(local_partial(start, count) if count > 0 else None)
    ref = next((P for P in mine if P is not None), None)
    dev = ref.device if ref is not None else (torch.device(device) if device is not None else torch.device("cpu"))
    block = torch.stack([(P if P is not None else torch.eye(d, dtype=torch.complex128, device=dev)).contiguous()
                         for P in mine])
    t = block.view(torch.float64)
    gathered = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(gathered, t, group=group)
    parts = []
    for r in range(world):
        g = gathered[r].view(torch.complex128)
        for v in range(virtual):
            parts.append(g[v] if ranges[r * virtual + v][1] > 0 else None)
    return combine_partials(parts, mul)


def sharded_state(local_partial: Callable, N: int, d: int, psi0, apply: Callable, group=None):
    """State form of the interval sharding.  Every rank calls this with the same N, d and
    psi0 (a complex128 tensor on the rank's device): it forms its own range's partial
    product with local_partial(start, count) (all ranks at once), then the state passes from
    rank to rank in time order (rank r receives psi_r, forms psi_{r+1} = apply(P_r, psi_r),
    sends it on; a rank with an empty range passes psi on), and the last rank broadcasts
    psi(T), which every rank returns."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)

    def glob(r):
        return r if group is None else dist.get_global_rank(group, r)

    start, count = interval_ranges(N, world)[rank]
    P = local_partial(start, count) if count > 0 else None
    buf = torch.empty(2 * d, dtype=torch.float64, device=psi0.device)
    if rank == 0:
        psi = psi0.clone()
    else:
        dist.recv(buf, src=glob(rank - 1), group=group)
        psi = buf.view(torch.complex128).clone()
    if P is not None:
        psi = apply(P, psi)
    if rank < world - 1:
        dist.send(psi.contiguous().view(torch.float64), dst=glob(rank + 1), group=group)
    else:
        buf.copy_(psi.contiguous().view(torch.float64))
    dist.broadcast(buf, src=glob(world - 1), group=group)
    return buf.view(torch.complex128).clone()


def max_over_ranks(value: float, group=None, device=None) -> float:
    """The slowest rank's time (what a multi-GPU step costs)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


# ----------------------------------------------------------------------------
# the GPU form: partials by mg_evolve, the combination by mg_cgemm
# ----------------------------------------------------------------------------
def evolve_propagator_sharded(ctx, H0, Hk, samples, N: int, P: int, t0: float, dt: float, w,
                              precision: Optional[int] = None, slices: int = 6, group=None, virtual: int = 1,
                              reorth_every: int = 0, plan=None):
    """U(T) of one job whose N intervals are shared by the ranks of `group` (each on its own
    GPU, ctx that GPU's context): every rank evolves its ranges through mg_set_controls /
    mg_evolve (samples: the job's N x P x K drive samples on this device; a range takes its
    rows and starts at t0 + start dt), the partials are all-gathered (NCCL), and every rank
    multiplies them in time order with mg_cgemm on its GPU.  Returns the d x d device tensor.
    `plan` (optional) is a Plan of H0, H_k in this precision to reuse across calls (else one
    is made and freed here)."""
    import torch
    from . import magnus as M
    prec = M.MG_PREC_SPLIT if precision is None else precision
    d = int(H0.shape[0])
    dev = samples.device
    own = plan is None
    if own:
        plan = M.Plan(ctx, H0, Hk, prec, slices)

    def local_partial(start, count):
        plan.set_controls(count, P, t0 + start * dt, dt, w, samples[start:start + count].contiguous())
        out = torch.empty((d, d), dtype=torch.complex128, device=dev)
        plan.evolve(M.MG_OUT_PROPAGATOR, None, out, reorth_every, report=False)
        torch.cuda.current_stream(dev).synchronize()
        if ctx.stream is not None:
            ctx.stream.synchronize()
        return out

    def mul(A, B):
        C = torch.empty_like(A)
        M.mg_cgemm(ctx, 1, d, A.contiguous(), B.contiguous(), C, prec, slices)
        if ctx.stream is not None:
            ctx.stream.synchronize()
        return C

    try:
        return sharded_propagator(local_partial, N, d, mul, group=group, virtual=virtual, device=dev)
    finally:
        if own:
            plan.close()
