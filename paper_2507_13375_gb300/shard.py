"""One layer-assignment round split over several GPUs by nets (host logic).

Within a round every net sees the same snapshot (D, H) (Alg. 2: one batch
against one demand map), so the nets split into contiguous ranges, one per
GPU (one process and one library context each), with a single exchange per
round: the sum of the shards' int32 demand maps.  Every shard then applies
the same history update and penalty prefix (la_commit_demand), so all of
them enter the next round with the same snapshot.  The Elmore passes and the
adjoint reweighting are per net and need no exchange.

The functions here only split ranges and order the calls; the arithmetic of
the round runs in the library's kernels on each GPU.
"""
from __future__ import annotations

import numpy as np
import torch


def shard_ranges(net_ptr, world: int):
    """Contiguous net ranges [lo, hi), one per rank, of about V / world nodes
    each: rank r starts at the first net whose first node is at or after
    r V / world.  Every range holds at least one net (needs N >= world)."""
    net_ptr = np.asarray(net_ptr, dtype=np.int64)
    N, V = len(net_ptr) - 1, int(net_ptr[-1])
    if world < 1 or N < world:
        raise ValueError(f"cannot split {N} nets over {world} shards")
    cuts = [0]
    for r in range(1, world):
        c = int(np.searchsorted(net_ptr[:N], (r * V) // world, side="left"))
        cuts.append(min(max(c, cuts[-1] + 1), N - (world - r)))
    cuts.append(N)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard_forest(forest: dict, lo: int, hi: int) -> dict:
    """The nets [lo, hi) of a forest as a forest of their own (node ids and
    net pointers renumbered from 0)."""
    ptr = np.asarray(forest["net_ptr"], dtype=np.int64)
    a, b = int(ptr[lo]), int(ptr[hi])
    out = {k: forest[k][a:b] for k in ("x", "y", "parent", "pin_layer", "sink_cap", "kappa")}
    out["net_ptr"] = ptr[lo:hi + 1] - a
    out["r_drv"] = forest["r_drv"][lo:hi]
    out["num_nets"], out["num_nodes"] = hi - lo, b - a
    return out


def sharded_round(shard, allreduce_sum, **round_kwargs) -> dict:
    """One round of a forest split by nets: this shard's DP, backtrack and
    demand (local_demand), the sum of every shard's demand (`allreduce_sum`,
    in place on a tensor), and la_commit_demand.  `shard` is a LayerAssigner
    (or anything with its assign_round / get_state / commit_demand calls).
    Returns the round's statistics for the whole forest: tof and the ReLU
    overflow from the summed map, J, vias and wirelength summed over shards."""
    st = shard.assign_round(local_demand=True, **round_kwargs)
    D, _ = shard.get_state()
    allreduce_sum(D)
    cm = shard.commit_demand(D)
    out = dict(st) if st else {}
    if st is not None:
        dev = D.device if isinstance(D, torch.Tensor) else "cpu"
        tot = torch.tensor([float(st["total_cost"]), float(st["vias"]), float(st["wl"])], dtype=torch.float64,
                           device=dev)
        allreduce_sum(tot)
        out.update(total_cost=float(tot[0]), vias=int(tot[1]), wl=int(tot[2]), tof=cm["tof"],
                   relu_overflow=cm["relu_overflow"], local_total_cost=float(st["total_cost"]))
    return out
