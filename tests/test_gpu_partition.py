"""The partitioned step through the library (paper_1903_11521_gb300.partition.PartitionedSolver):
two gloo ranks on cuda:0, each holding its block of elements, the halo of remote face
projections gathered by the library (yt_solver_halo_pack), staged through host memory,
received into the halo block (yt_solver_halo_unpack), the neighbour kernel run on the
tiles without remote neighbours first and on the others after the exchange.  The
processes exchange only on the host between kernel launches (no kernel waits for the
other process).  The gathered result equals the single-solver step bitwise (every
element is computed from the same inputs by the same code) and the oracle to 1e-12."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import parity
import workload as wl
from oracle import basis, scheme

pytestmark = pytest.mark.gpu
ORDER = 4
STEPS = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs(kind):
    if kind in ("random", "scattered"):
        E = 300
        el = wl.random_elements(E, seed=310)
        conn = wl.random_connectivity(E, seed=311)
    else:
        mesh = wl.jittered_periodic_mesh(4, jitter=0.1, seed=312)
        el, conn = mesh.elements, mesh.conn
    E = el.rho.size
    Q = wl.random_dofs(E, basis.n_basis(ORDER - 1), seed=313, scale="impedance", elements=el)
    dt = wl.cfl_time_step(el, ORDER - 1)
    return el, conn, Q, dt


def _owner(E, world, kind):
    if kind == "scattered":
        # every rank's elements spread over the mesh: the solver's own order differs from
        # the global one, and most tiles have remote faces
        return np.random.default_rng(314).permutation(np.arange(E) % world)
    from paper_1903_11521_gb300 import partition
    return partition.block_partition(E, world)


def _rank(rank, world, port, kind, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1903_11521_gb300 as yt
    from paper_1903_11521_gb300 import partition
    el, conn, Q, dt = _inputs(kind)
    owner = _owner(el.rho.size, world, kind)
    ps = partition.PartitionedSolver(ORDER, dt, el, conn, owner, rank, dist, precision=yt.YT_F64,
                                     staging="host")
    ps.set_dofs(Q)
    for _ in range(STEPS):
        ps.step()
    ids, q = ps.get()
    info = (ps.n_interior_tiles, ps.n_tiles, ps.n_halo)
    ps.close()
    gathered = [None] * world if rank == 0 else None
    dist.gather_object((ids, q, info), gathered, dst=0)
    if rank == 0:
        full = np.zeros_like(Q)
        infos = []
        for ids_r, q_r, info_r in gathered:
            full[ids_r] = q_r
            infos.append(info_r)
        np.save(out_path, full)
        np.save(out_path + ".info.npy", np.array(infos))
    dist.destroy_process_group()


@pytest.mark.timeout(600)
@pytest.mark.parametrize("kind", ["random", "structured", "scattered"])
def test_two_rank_partitioned_step(tmp_path, kind):
    import paper_1903_11521_gb300 as yt
    out = str(tmp_path / "full.npy")
    mp.start_processes(_rank, args=(2, _free_port(), kind, out), nprocs=2, join=True,
                       start_method="spawn")
    full = np.load(out)
    infos = np.load(out + ".info.npy")
    print(f"PARITY partitioned {kind}: (interior tiles, tiles, halo slots) per rank {infos.tolist()}")
    assert (infos[:, 2] > 0).all()                    # both ranks receive a halo
    el, conn, Q, dt = _inputs(kind)
    s = yt.Solver(ORDER, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, conn.neighbours,
                  conn.faces, conn.orient)
    s.set_dofs_host(Q)
    for _ in range(STEPS):
        s.step()
    single = s.get_host()
    s.close()
    assert np.array_equal(full, single)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref = Q
    for _ in range(STEPS):
        ref, _ = scheme.ader_step(ref, star, loc, nb, conn.neighbours, conn.faces, conn.orient, dt,
                                  ORDER - 1)
    parity.check(f"partitioned {kind} f64 {STEPS} steps Q", full, ref, parity.F64, parity.F64)
    if kind == "structured":
        assert (infos[:, 0] > 0).all()                # interior tiles ran before the exchange
