"""Element partition and halo exchange for a multi-GPU step (host logic).

The step shards by elements: after the local kernel every rank holds the face
projections R^jT I of its own elements; the neighbour kernel of an element whose face
neighbour lives on another rank needs that neighbour's projection for face j.  This is
the only data exchanged per step (B~ x 9 values per remote face), once per step.

Every rank knows the global connectivity, so both sides of an exchange derive the same
ordered lists without negotiation: rank r receives, from each peer p, the projections of
the (element, face) pairs of p's elements that r's elements touch, in increasing
(element, face) order, and sends the mirror lists.  Received projections form a halo
block appended after the rank's own elements; the rank's connectivity is rewritten to
local indices (own elements) or halo slots.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def block_partition(n_elements: int, n_parts: int) -> np.ndarray:
    """Owner rank of every element: contiguous blocks of nearly equal size."""
    return np.minimum(np.arange(n_elements, dtype=np.int64) * n_parts // n_elements, n_parts - 1)


@dataclass
class HaloPlan:
    rank: int
    local: np.ndarray                      # global ids of the rank's elements, increasing
    recv: dict = field(default_factory=dict)   # peer -> array of (global element, face j)
    send: dict = field(default_factory=dict)   # peer -> array of (local index, face j)
    neighbour_slot: np.ndarray = None      # (n_local, 4): local index, or n_local + halo slot
    neighbour_face: np.ndarray = None      # (n_local, 4): j of the neighbour's projection


def halo_plan(owner: np.ndarray, neighbours: np.ndarray, faces: np.ndarray, rank: int) -> HaloPlan:
    owner = np.asarray(owner)
    local = np.nonzero(owner == rank)[0]
    g2l = -np.ones(owner.shape[0], dtype=np.int64)
    g2l[local] = np.arange(local.size)
    plan = HaloPlan(rank=rank, local=local)
    # what this rank needs: remote (element, face) pairs referenced by its elements
    nb = neighbours[local]
    fj = faces[local]
    remote = owner[nb] != rank
    pairs = sorted({(int(g), int(j)) for g, j in zip(nb[remote], fj[remote])})
    slot = {}
    halo = 0
    for peer in sorted(set(int(owner[g]) for g, _ in pairs)):
        lst = [(g, j) for g, j in pairs if owner[g] == peer]
        plan.recv[peer] = np.array(lst, dtype=np.int64).reshape(-1, 2)
        for p in lst:
            slot[p] = halo
            halo += 1
    # what peers need from this rank: pairs (own element, face) referenced by their elements
    others = np.nonzero(owner != rank)[0]
    onb = neighbours[others]
    ofj = faces[others]
    mine = owner[onb] == rank
    for peer in sorted(set(int(x) for x in owner[others][np.any(mine, axis=1)])):
        sel = owner[others] == peer
        m = mine & sel[:, None]
        lst = sorted({(int(g), int(j)) for g, j in zip(onb[m], ofj[m])})
        plan.send[peer] = np.array([(g2l[g], j) for g, j in lst], dtype=np.int64).reshape(-1, 2)
    n_local = local.size
    plan.neighbour_slot = np.where(remote, 0, g2l[nb])
    plan.neighbour_face = fj.copy()
    for e in range(n_local):
        for s in range(4):
            if remote[e, s]:
                plan.neighbour_slot[e, s] = n_local + slot[(int(nb[e, s]), int(fj[e, s]))]
    return plan


def exchange(plan: HaloPlan, projections: np.ndarray, dist=None) -> np.ndarray:
    """projections: (n_local, 4, Bt, 9) of the rank's elements.  Returns the halo block
    (n_halo, Bt, 9) in slot order.  `dist` is torch.distributed (any backend); sends and
    receives are posted together and waited for once."""
    import torch
    if dist is None:
        import torch.distributed as dist
    bt, nq = projections.shape[2], projections.shape[3]
    reqs, recv_bufs = [], {}
    for peer, lst in plan.recv.items():
        buf = torch.empty((lst.shape[0], bt, nq), dtype=torch.float64)
        recv_bufs[peer] = buf
        reqs.append(dist.irecv(buf, src=peer))
    for peer, lst in plan.send.items():
        data = torch.from_numpy(np.ascontiguousarray(projections[lst[:, 0], lst[:, 1]]))
        reqs.append(dist.isend(data, dst=peer))
    for r in reqs:
        r.wait()
    if not recv_bufs:
        return np.zeros((0, bt, nq))
    return np.concatenate([recv_bufs[p].numpy() for p in sorted(recv_bufs)])
