"""Host logic of the partitioned step (paper_1903_11521_gb300.partition) with two and three
gloo ranks on CPU, element blocks and scattered owners: each rank computes its elements' face projections, exchanges the remote
ones, applies the neighbour flux with local + halo projections, and the gathered result
equals the oracle's single-process step.  The per-element arithmetic here uses the
oracle's factorised matrices (this is a test of the partition and exchange logic)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workload as wl
from oracle import basis, scheme
from paper_1903_11521_gb300 import partition

ORDER_N = 2
E = 60


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    el = wl.random_elements(E, seed=300)
    conn = wl.random_connectivity(E, seed=301)
    Q = wl.random_dofs(E, basis.n_basis(ORDER_N), seed=302, scale="impedance", elements=el)
    dt = wl.cfl_time_step(el, ORDER_N)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    return el, conn, Q, dt, star, loc, nb


def _owner(world, kind):
    if kind == "block":
        return partition.block_partition(E, world)
    # scattered owners: every rank's elements spread over the mesh
    return np.random.default_rng(303 + world).permutation(np.arange(E) % world)


def _rank(rank, world, port, out_path, kind="block"):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    el, conn, Q, dt, star, loc, nb = _inputs()
    m = basis.float_matrices(ORDER_N)
    owner = _owner(world, kind)
    plan = partition.halo_plan(owner, conn.neighbours, conn.faces, rank)
    mine = plan.local
    # local phase of the own elements
    _, I = scheme.derivatives_and_time_integral(Q[mine], star[mine], dt, ORDER_N)
    Qloc = scheme.local_update(Q[mine], I, star[mine], loc[mine], ORDER_N)
    proj = np.stack([np.einsum('lm,elq->emq', m['R'][j], I) for j in range(4)], axis=1)
    halo = partition.exchange(plan, proj, dist)
    allproj = np.concatenate([proj, np.zeros((halo.shape[0], 4) + proj.shape[2:])])
    # neighbour phase: projection of the neighbour's face j, local or from the halo
    out = Qloc.copy()
    for e in range(mine.size):
        g = mine[e]
        for s in range(4):
            slot, j, h = plan.neighbour_slot[e, s], conn.faces[g, s], conn.orient[g, s]
            P = allproj[slot, j] if slot < mine.size else halo[slot - mine.size]
            out[e] += m['Rhat'][s] @ m['f'][h] @ P @ nb[g, s].T
    gathered = [None] * world if rank == 0 else None
    dist.gather_object((mine, out), gathered, dst=0)
    if rank == 0:
        full = np.zeros_like(Q)
        for ids, vals in gathered:
            full[ids] = vals
        np.save(out_path, full)
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["block", "scattered"])
def test_halo_plan_is_consistent(kind):
    _, conn, _, _, _, _, _ = _inputs()
    owner = _owner(3, kind)
    plans = [partition.halo_plan(owner, conn.neighbours, conn.faces, r) for r in range(3)]
    for r, p in enumerate(plans):
        for peer, lst in p.recv.items():
            sent = plans[peer].send[r]
            # the peer sends exactly what r receives, in the same order
            assert np.array_equal(plans[peer].local[sent[:, 0]], lst[:, 0])
            assert np.array_equal(sent[:, 1], lst[:, 1])
        assert np.all(p.neighbour_slot < p.local.size + sum(len(v) for v in p.recv.values()))


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world, kind", [(2, "block"), (3, "scattered")])
def test_multi_rank_step_equals_single_process(tmp_path, world, kind):
    out = str(tmp_path / "full.npy")
    mp.start_processes(_rank, args=(world, _free_port(), out, kind), nprocs=world, join=True,
                       start_method="spawn")
    full = np.load(out)
    el, conn, Q, dt, star, loc, nb = _inputs()
    ref, _ = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient, dt,
                              ORDER_N)
    assert np.allclose(full, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
