"""Energy terms split across ranks (one process per GPU).

The networks of an energy evaluation -- the norm and every local term, or
the two cluster networks of every term (Sec. V) -- are independent
contractions, so rank r contracts networks r, r + world, r + 2 world, ...
(strided, which spreads the uneven term sizes) and nothing else.  The only
exchange is one all-reduce of the (mantissa, log-scale) pairs of all
networks, each of which exactly one rank has filled in (the others hold
zeros, so the FP64 sum reproduces every value bit for bit).  Every rank then
calls the same ftn_energy_reduce on the same values, so the energy equals
the single-process result exactly.  Marshalling only: contractions and the
reduction run in libftn; torch.distributed carries the values (gloo on the
host, NCCL between GPUs).
"""
from __future__ import annotations

from . import ftn


def shard(count, rank, world):
    """Indices of the networks rank ``rank`` of ``world`` contracts."""
    return list(range(rank, count, world))


def gather_values(count, idx, values, device=None):
    """All networks' (mantissa, log_scale) on every rank, from each rank's
    values for its indices ``idx``."""
    import torch
    import torch.distributed as dist

    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    buf = torch.zeros((max(count, 1), 2), dtype=torch.float64, device=device)
    if idx:
        buf[idx] = torch.tensor([[float(m), float(lg)] for m, lg in values], dtype=torch.float64, device=device)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    host = buf.cpu().tolist()
    return [(host[i][0], host[i][1]) for i in range(count)]


def energy_sharded(networks, num, den, group_end, rank, world, contract, device=None):
    """Energies per group and term ratios of ``networks`` with this rank
    contracting its share.  ``contract(list of networks)`` returns their
    (mantissa, log_scale) values -- e.g. ``lambda nets: ftn.energy(ctxs,
    nets, [], [], [], prec)[2]``.  Returns (energies, ratios)."""
    nets = list(networks)
    idx = shard(len(nets), rank, world)
    local = contract([nets[i] for i in idx]) if idx else []
    values = gather_values(len(nets), idx, local, device) if world > 1 else local
    return ftn.energy_reduce(values, num, den, group_end)
