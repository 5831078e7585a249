"""Element partitions and the interface exchange of a distributed Q^T (host logic).

The paper's codes distribute elements over ranks; the direct-stiffness sum of
Eq. (36) then has an on-rank part and an exchange of interface-node sums
between neighbouring ranks (Sec. 8.2 describes the two stages for the GPU code:
an on-device condense of the shared nodes, then a host-staged exchange).

This module holds the partition-ready data structures for that split:

* ``partition_slabs`` -- contiguous slabs of the element array along z;
* ``Plan`` -- for each rank its nodes, the owned subset (each global node is
  owned by the lowest rank touching it) and the interface subset (nodes touched
  by more than one rank) with the ranks sharing each;
* ``exchange_sum`` -- completes a rank-local partial sum over the rank's nodes
  into the global sum on its interface nodes through ``torch.distributed``
  (one all-reduce over the union of interface nodes, in a fixed order).

Solves on the GPU run as independent replicas (one per rank), so this exchange is
exercised on CPU ranks (gloo); it is the stage a multi-GPU solve would insert
between the element kernel and the vector update.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def partition_slabs(Ex: int, Ey: int, Ez: int, nparts: int) -> list[np.ndarray]:
    """Element ids (e = ex + Ex (ey + Ey ez)) of nparts contiguous z-slabs."""
    if not 1 <= nparts <= Ez:
        raise ValueError("need 1 <= nparts <= Ez")
    bounds = np.linspace(0, Ez, nparts + 1).round().astype(int)
    per_layer = Ex * Ey
    return [np.arange(bounds[p] * per_layer, bounds[p + 1] * per_layer, dtype=np.int64) for p in range(nparts)]


@dataclass
class Plan:
    nodes: list[np.ndarray]        # sorted global nodes touched by each rank
    owned: list[np.ndarray]        # nodes each rank owns (lowest touching rank)
    interface: np.ndarray          # sorted global nodes touched by two or more ranks
    sharers: dict[int, list[int]]  # interface node -> ranks touching it


def build_plan(l2g_parts: list[np.ndarray]) -> Plan:
    """Plan from each rank's l2g rows ([E_r, p1^3] global ids)."""
    nodes = [np.unique(np.asarray(l).reshape(-1)) for l in l2g_parts]
    touch: dict[int, list[int]] = {}
    for r, nd in enumerate(nodes):
        for g in nd.tolist():
            touch.setdefault(g, []).append(r)
    interface = np.array(sorted(g for g, rs in touch.items() if len(rs) > 1), dtype=np.int64)
    owned = [np.array(sorted(g for g in nd.tolist() if touch[g][0] == r), dtype=np.int64)
             for r, nd in enumerate(nodes)]
    return Plan(nodes=nodes, owned=owned, interface=interface,
                sharers={int(g): touch[int(g)] for g in interface.tolist()})


def exchange_sum(partial: np.ndarray, rank: int, plan: Plan, dist) -> np.ndarray:
    """partial[i] = this rank's contribution at plan.nodes[rank][i]; returns the
    global sums at the same nodes (interface entries summed over all ranks)."""
    import torch
    nodes = plan.nodes[rank]
    pos = np.searchsorted(plan.interface, nodes)
    on_if = (pos < len(plan.interface)) & (plan.interface[np.minimum(pos, len(plan.interface) - 1)] == nodes)
    buf = np.zeros(len(plan.interface), dtype=np.float64)
    buf[pos[on_if]] = partial[on_if]
    t = torch.from_numpy(buf)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = np.array(partial, dtype=np.float64, copy=True)
    out[on_if] = t.numpy()[pos[on_if]]
    return out
