"""One (T) energy over the ranks of a torch.distributed group.

Each rank computes its contiguous range of the occupied triplets on its own
device (tc_energy_shard_dev: the range, the kernels and the rank's
compensated (sum, compensation) pair all come from libtc).  The one exchange
is an all_gather of these pairs; tc_combine_parts adds them in rank order, so
every rank holds the same E_(T) bits whatever order the collective used.
This module only moves the pairs between processes.
"""
from __future__ import annotations

import paper_2512_01055_gb300 as tc


def gather_parts(part, group=None):
    """All ranks' (sum, compensation) pairs, in rank order (one all_gather of two doubles per rank)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    mine = torch.tensor(list(part), dtype=torch.float64, device=dev)
    out = [torch.empty(2, dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(out, mine, group=group)
    return [tuple(x.cpu().tolist()) for x in out]


def energy(ctx, o, v, eps, t1, t2, ovvv, ovoo, ovov, prec=tc.TC_FP64, slices=0, group=None, stream=None):
    """E_(T) of one job split over the group's ranks; every rank passes its own device copy of the inputs.

    Returns (E_(T), this rank's tc_result); E_(T) is bitwise the same on every rank.
    """
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    part, res = tc.tc_energy_shard_dev(ctx, o, v, eps, t1, t2, ovvv, ovoo, ovov, rank, world, prec=prec,
                                       slices=slices, stream=stream)
    return tc.tc_combine_parts(gather_parts(part, group)), res
