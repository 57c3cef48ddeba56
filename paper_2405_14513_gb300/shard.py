"""One field's estimate split over the ranks of a process group.

Every rank holds a plan of the same description and the same input field;
rank r runs share r of the Step-II work (``Plan.estimate_part``) and one
sum all-reduce of the FP64 output completes the estimate on every rank: the
numerator of Eq. bs_lm2_1 is a sum over combinations, so the shares'
outputs add up to the whole (NaN bins stay NaN).  The transforms and Step I
run whole on every rank (a few per cent of the work at 512^3), so nothing
but the 1.5 MB output (512^3, 30 k1 bins) crosses between devices.
"""
from __future__ import annotations


def estimate_sharded(plan, delta, workspace, out=None, group=None, stream=None):
    """Share dist.get_rank(group) of dist.get_world_size(group) of
    plan.estimate(delta), then a SUM all-reduce of the output in place.
    Returns the whole estimate (the same tensor on every rank)."""
    import torch
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    out = plan.estimate_part(delta, workspace, rank, world, out=out, stream=stream)
    if out.is_cuda and stream is not None:
        # the collective runs after the share on the caller's stream
        torch.cuda.current_stream(out.device).wait_stream(stream)
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out
