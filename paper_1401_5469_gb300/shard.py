"""One Monte Carlo iteration of one model split across processes (one GPU
each): disjoint packet ranges, then a sum of the estimators.

Packet draws are keyed by (seed, packet index, iteration), so the packets of
rank r -- the contiguous range packet_range(r, world, N) -- are exactly the
packets that index range would carry in a single-GPU run, and the summed
J_est, nu_bar, J_blue and spectrum are the single-GPU iteration's sums up to
summation order.  The sum is the only exchange (Sect. 2.8 needs all packets'
estimators before the T_R/W update); every rank then applies Eqs. 15-16 to
identical sums, so the plasma state stays identical on every rank without
further communication.
"""
from __future__ import annotations


def packet_range(rank: int, world: int, n_packets: int):
    """(first, count) of rank's contiguous share; the shares tile [0, n)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, rem = divmod(int(n_packets), world)
    first = rank * base + min(rank, rem)
    return first, base + (1 if rank < rem else 0)


def run_sharded_iteration(model, seed: int, iteration: int, n_packets: int, t_inner: float,
                          group=None, j_blue: bool = False, update: bool = True):
    """Run this rank's packets of the iteration, sum the estimators across the
    group in place on the device, then (if `update`) apply the T_R/W update.

    `model` provides run_iteration_range, synchronize, device_estimators and
    update_radiation_field (mc.Model does).  Needs n_packets >= world size so
    that every rank's range is non-empty."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    if n_packets < world:
        raise ValueError("need at least one packet per rank")
    first, count = packet_range(rank, world, n_packets)
    model.run_iteration_range(seed, iteration, first, count, n_packets, t_inner)
    model.synchronize()  # the sums are complete on the model's stream
    views = model.device_estimators()
    names = ["j_est", "nu_bar", "spectrum"] + (["j_blue"] if j_blue and views["j_blue"] is not None else [])
    for n in names:
        dist.all_reduce(views[n], op=dist.ReduceOp.SUM, group=group)
    _sync_device(views["j_est"])
    if update:
        return model.update_radiation_field()
    return None


def _sync_device(t):
    if t.is_cuda:
        import torch
        torch.cuda.current_stream(t.device).synchronize()
