"""Channel sharding across GPUs (one process per GPU, no collective).

Channels are independent, so a batch shards by channel with no exchange: rank
r filters a contiguous range of channels whose summed cost -- samples times
the method's FMAs per sample, len_c (6 K_c + 1), or the HBM bytes when those
dominate -- is as close as possible to 1 / world of the total.  Contiguous
ranges keep each rank's slice of the packed signals one contiguous span.
Only the host computes the split; no data moves between ranks.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch


def channel_costs(lengths: Sequence[int], K: Sequence[int], bytes_weight: float = 0.0
                  ) -> List[float]:
    """Per channel, len (6 K + 1) FMAs plus bytes_weight x 8 bytes per sample
    (bytes_weight: FMA time per byte, to weigh HBM-bound channels)."""
    return [float(n) * (6 * int(k) + 1 + 8.0 * bytes_weight) for n, k in zip(lengths, K)]


def partition_by_cost(costs: Sequence[float], world: int) -> List[Tuple[int, int]]:
    """Contiguous channel ranges [c0, c1) per rank, cut where the prefix cost
    crosses r / world of the total (every rank gets a range, possibly empty
    when there are fewer channels than ranks)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    C = len(costs)
    total = float(sum(costs))
    bounds = [0]
    acc = 0.0
    c = 0
    for r in range(1, world):
        target = total * r / world
        while c < C and acc + costs[c] / 2.0 <= target:
            acc += costs[c]
            c += 1
        bounds.append(max(c, bounds[-1]))
    bounds.append(C)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def shard(x: torch.Tensor, sos: torch.Tensor, K: torch.Tensor, lengths: Sequence[int],
          zi, c0: int, c1: int):
    """The packed slices of one rank's channels [c0, c1): (x, sos, K, lengths,
    zi) of that range (views where possible)."""
    lh = [int(v) for v in lengths]
    off0 = sum(lh[:c0])
    off1 = off0 + sum(lh[c0:c1])
    return (x[off0:off1], sos[c0:c1], K[c0:c1], lh[c0:c1],
            zi[c0:c1] if zi is not None else None)
