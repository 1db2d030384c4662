"""Element partition and halo exchange of a multi-GPU step.

The step shards by elements: after the local kernel every rank holds the face
projections R^jT I of its own elements; the neighbour kernel of an element whose face
neighbour lives on another rank needs that neighbour's projection for face j.  This is
the only data exchanged per step (B~ x 9 values per remote face), once per step.

Every rank knows the global connectivity, so both sides of an exchange derive the same
ordered lists without negotiation: rank r receives, from each peer p, the projections of
the (element, face) pairs of p's elements that r's elements touch, in increasing
(element, face) order, and sends the mirror lists.  Received projections form a halo
block after the rank's own elements; the rank's connectivity is rewritten to local
indices (own elements) or halo slots.

PartitionedSolver runs this with the library: its own elements ordered with the ones
without a remote neighbour first, so that the neighbour kernel of those tiles runs while
the halo is in flight (yt_step_phase_tiles), the halo gathered by yt_solver_halo_pack and
received into the library's halo block (yt_solver_halo_unpack); the transfer itself goes
through torch.distributed (NCCL device buffers, or host staging for gloo).
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
    E = owner.shape[0]
    local = np.nonzero(owner == rank)[0]
    g2l = -np.ones(E, dtype=np.int64)
    g2l[local] = np.arange(local.size)
    plan = HaloPlan(rank=rank, local=local)
    # what this rank needs: remote (element, face) pairs referenced by its elements, as
    # codes 4 g + j, unique and increasing (= increasing (g, j))
    nb = neighbours[local].astype(np.int64)
    fj = faces[local].astype(np.int64)
    remote = owner[nb] != rank
    codes = np.unique(4 * nb[remote] + fj[remote])
    peers_of = owner[codes // 4]
    order = np.argsort(peers_of, kind="stable")      # by peer, (g, j) increasing within
    codes = codes[order]
    peers_of = peers_of[order]
    for peer in np.unique(peers_of):
        c = codes[peers_of == peer]
        plan.recv[int(peer)] = np.stack([c // 4, c % 4], axis=1)
    # what peers need from this rank: pairs (own element, face) referenced by theirs
    others = np.nonzero(owner != rank)[0]
    onb = neighbours[others].astype(np.int64)
    ofj = faces[others].astype(np.int64)
    mine = owner[onb] == rank
    peer_rows = np.broadcast_to(owner[others][:, None], onb.shape)
    for peer in np.unique(peer_rows[mine]):
        sel = mine & (peer_rows == peer)
        c = np.unique(4 * onb[sel] + ofj[sel])
        plan.send[int(peer)] = np.stack([g2l[c // 4], c % 4], axis=1)
    n_local = local.size
    slot_of = np.empty(codes.size, dtype=np.int64)
    slot_of[:] = np.arange(codes.size)
    sorted_codes = np.argsort(codes)
    plan.neighbour_slot = np.where(remote, 0, g2l[nb])
    if codes.size:
        want = 4 * nb[remote] + fj[remote]
        pos = np.searchsorted(codes[sorted_codes], want)
        plan.neighbour_slot[remote] = n_local + slot_of[sorted_codes[pos]]
    plan.neighbour_face = fj.copy()
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


class PartitionedSolver:
    """One rank's part of a partitioned elastic step on the device (library kernels, one
    halo exchange per step).  `elements` / `conn` describe the whole mesh, `owner` the
    rank of every element.  staging="device": device buffers handed to dist (NCCL);
    "host": the halo goes through host memory (gloo)."""

    def __init__(self, order, dt, elements, conn, owner, rank, dist, precision=None, stream=None,
                 staging="device"):
        import torch

        from . import _lib
        from .solver import Solver
        self.dist, self.rank, self.stream, self.staging = dist, rank, stream, staging
        precision = _lib.YT_F64 if precision is None else precision
        plan = halo_plan(owner, conn.neighbours, conn.faces, rank)
        self.plan = plan
        n_local = plan.local.size
        remote = owner[conn.neighbours[plan.local]] != rank
        boundary = remote.any(axis=1)
        perm = np.concatenate([np.nonzero(~boundary)[0], np.nonzero(boundary)[0]])
        inv = np.empty(n_local, dtype=np.int64)
        inv[perm] = np.arange(n_local)
        self.ids = plan.local[perm]                       # global ids in the solver's order
        slot = plan.neighbour_slot[perm]
        nbr = np.where(slot < n_local, inv[np.minimum(slot, n_local - 1)], -1 - (slot - n_local))
        n_halo = int(sum(v.shape[0] for v in plan.recv.values()))
        self.n_interior_tiles = int((~boundary).sum()) // 32
        el = elements
        mat = np.stack([el.rho[self.ids], el.lam[self.ids], el.mu[self.ids]], axis=1)
        self.solver = Solver(order, dt, mat, el.jac[self.ids], nbr.astype(np.int32),
                             conn.faces[self.ids], conn.orient[self.ids], precision=precision,
                             stream=stream, n_halo=n_halo)
        self.n_tiles = (n_local + 31) // 32
        B_t = order * (order + 1) // 2
        self.row = 9 * B_t
        self.dtype = torch.float64 if precision == _lib.YT_F64 else torch.float32
        self.send_peers = sorted(plan.send)
        self.recv_peers = sorted(plan.recv)
        pairs = [np.stack([inv[plan.send[p][:, 0]], plan.send[p][:, 1]], axis=1) for p in self.send_peers]
        pairs = np.concatenate(pairs) if pairs else np.zeros((0, 2), dtype=np.int64)
        self.solver.set_send_list(pairs)
        self.send_counts = [plan.send[p].shape[0] for p in self.send_peers]
        self.recv_counts = [plan.recv[p].shape[0] for p in self.recv_peers]
        dev = "cuda"
        self.send_buf = torch.empty((max(1, pairs.shape[0]), self.row), dtype=self.dtype, device=dev)
        self.recv_buf = torch.empty((max(1, n_halo), self.row), dtype=self.dtype, device=dev)
        self.n_halo = n_halo

    def set_dofs(self, Q_global):
        """Q of the whole mesh (E, B, 9); this rank takes its elements."""
        self.solver.set_dofs_host(np.asarray(Q_global)[self.ids], stream=self.stream)

    def set_dofs_local(self, Q_local):
        """Q of this rank's elements (n_local, B, 9) in the solver's order (self.ids)."""
        self.solver.set_dofs_host(Q_local, stream=self.stream)

    def get(self):
        """(global ids, Q of this rank's elements (n_local, B, 9))."""
        return self.ids, self.solver.get_host(stream=self.stream)

    def _exchange(self):
        import torch
        dist = self.dist
        ops = []
        if self.staging == "host":
            torch.cuda.synchronize()
            send_h = self.send_buf.cpu()
            recv_h = torch.empty(self.recv_buf.shape, dtype=self.dtype)
            s0 = 0
            for p, n in zip(self.send_peers, self.send_counts):
                ops.append(dist.isend(send_h[s0:s0 + n].contiguous(), dst=p))
                s0 += n
            r0, views = 0, []
            for p, n in zip(self.recv_peers, self.recv_counts):
                v = torch.empty((n, self.row), dtype=self.dtype)
                views.append((r0, n, v))
                ops.append(dist.irecv(v, src=p))
                r0 += n
            for op in ops:
                op.wait()
            for r0, n, v in views:
                recv_h[r0:r0 + n] = v
            self.recv_buf.copy_(recv_h)
            return
        p2p = []
        s0 = 0
        for p, n in zip(self.send_peers, self.send_counts):
            p2p.append(dist.P2POp(dist.isend, self.send_buf[s0:s0 + n], p))
            s0 += n
        r0 = 0
        for p, n in zip(self.recv_peers, self.recv_counts):
            p2p.append(dist.P2POp(dist.irecv, self.recv_buf[r0:r0 + n], p))
            r0 += n
        if p2p:
            for w in dist.batch_isend_irecv(p2p):
                w.wait()

    def step(self):
        """One step: local kernel of all tiles, halo gather, neighbour kernel of the tiles
        without remote neighbours while the halo is exchanged, then of the others."""
        s = self.solver
        s.step_phase(0, stream=self.stream)
        if self.send_counts and sum(self.send_counts):
            s.halo_pack(self.send_buf.data_ptr(), stream=self.stream)
        s.step_phase_tiles(1, 0, self.n_interior_tiles, stream=self.stream)
        self._exchange()
        if self.n_halo:
            s.halo_unpack(self.recv_buf.data_ptr(), stream=self.stream)
        s.step_phase_tiles(1, self.n_interior_tiles, self.n_tiles - self.n_interior_tiles, stream=self.stream)

    def close(self):
        self.solver.close()
