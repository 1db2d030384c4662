"""Pins of the oracle's p-adaptive (mixed-order) step."""
import numpy as np

import workload as wl
from oracle import basis, planewave, scheme


def test_uniform_orders_reduce_to_plain_step():
    E, N = 20, 3
    el = wl.random_elements(E, seed=40)
    conn = wl.random_connectivity(E, seed=41)
    Q = wl.random_dofs(E, basis.n_basis(N), seed=42, scale="impedance", elements=el)
    dt = wl.cfl_time_step(el, N)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref, I = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, N)
    out, I2 = scheme.ader_step_mixed(list(Q), [N] * E, star, loc, nb, conn.neighbours,
                                     conn.faces, conn.orient, dt)
    assert np.allclose(np.array(out), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_mixed_orders_keep_constant_state_and_plane_wave_accuracy():
    """A constant state is preserved across order jumps; on a plane wave the mixed-order
    error lies between the errors of the lowest and highest uniform orders."""
    mesh = wl.periodic_cube_mesh(3)
    el = mesh.elements
    E = el.rho.size
    rng = np.random.default_rng(43)
    orders_n = rng.integers(1, 4, E)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    dt = wl.cfl_time_step(el, 3, cfl=0.3)
    Qc = [np.zeros((basis.n_basis(int(n)), 9)) for n in orders_n]
    for q in Qc:
        q[0, :] = np.arange(1, 10)
    out, _ = scheme.ader_step_mixed(Qc, orders_n, star, loc, nb, mesh.conn.neighbours,
                                    mesh.conn.faces, mesh.conn.orient, dt)
    assert max(np.abs(a - b).max() for a, b in zip(out, Qc)) < 1e-12 * 9
    k = 2 * np.pi * np.array([1.0, 1.0, 0.0])
    steps = 6
    errs = {}
    for label, ords in (("low", np.full(E, 1)), ("high", np.full(E, 3)), ("mixed", orders_n)):
        Q3 = planewave.project(mesh, 3, 0.0, k, 1.0, 2.0, 1.0)
        Q = [Q3[e, :basis.n_basis(int(ords[e]))] for e in range(E)]
        for _ in range(steps):
            Q, _ = scheme.ader_step_mixed(Q, ords, star, loc, nb, mesh.conn.neighbours,
                                          mesh.conn.faces, mesh.conn.orient, dt)
        full = np.zeros((E, basis.n_basis(3), 9))
        for e in range(E):
            full[e, :Q[e].shape[0]] = Q[e]
        errs[label] = planewave.l2_error(mesh, 3, full, steps * dt, k, 1.0, 2.0, 1.0)[6]
    assert errs["high"] < errs["mixed"] < errs["low"]
