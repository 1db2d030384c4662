"""Pins of the 27-quantity viscoelastic-shaped oracle (oracle/viscoelastic.py).

The paper gives no equations for the rheology, so physics is not pinned; what is pinned
is that the oracle computes the stated system: its Jacobians and flux solvers against
their eigenstructure, the reduction to the elastic oracle without the source, the pure
source step against the closed-form solution of the relaxation ODE, a constant state on a
periodic mesh (volume and fluxes cancel, only the source acts) and linearity."""
from math import factorial

import numpy as np
import pytest

import workload as wl
from oracle import basis, scheme
from oracle import viscoelastic as ve


def _case(E, order_n, seed):
    el = wl.random_elements(E, seed=seed)
    conn = wl.random_connectivity(E, seed=seed + 1)
    dt = wl.cfl_time_step(el, order_n)
    att = wl.attenuation(el, dt, seed=seed + 2)
    Q = wl.random_dofs_viscoelastic(E, basis.n_basis(order_n), el, att, seed=seed + 3)
    return el, conn, dt, att, Q


def _setup(el, att):
    return ve.setup_element_matrices(el.rho, el.lam, el.mu, att.ylam, att.ymu, att.omega, el.jac)


def test_jacobian_structure_and_spectrum():
    el, _, dt, att, _ = _case(5, 3, 11)
    A, Bm, C = ve.jacobians(el.rho, el.lam, el.mu, att.ylam, att.ymu, att.omega)
    elastic = scheme.elastic_jacobians(el.rho, el.lam, el.mu)
    for J, Je in zip((A, Bm, C), elastic):
        assert np.array_equal(J[:, :9, :9], Je)
        assert not J[:, :, 9:].any()                     # anelastic functions carry no flux
        assert not J[:, 9:, :6].any()                    # they are driven by velocities only
        assert J[:, 9:, 6:9].any()
    # the anelastic rows of mechanism l are omega_l times the stress rows with Y_l moduli
    for l in range(3):
        ref = scheme.elastic_jacobians(el.rho, att.ylam[:, l], att.ymu[:, l])[0][:, :6, 6:9]
        r0 = ve.theta_index(l, 0)
        assert np.allclose(A[:, r0:r0 + 6, 6:9], att.omega[:, l, None, None] * ref, rtol=1e-15)
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    An = n[0] * A + n[1] * Bm + n[2] * C
    cp = np.sqrt((el.lam + 2 * el.mu) / el.rho)
    cs = np.sqrt(el.mu / el.rho)
    for e in range(5):
        ev = np.sort(np.linalg.eigvals(An[e]).real)
        expect = np.sort(np.concatenate([[-cp[e], -cs[e], -cs[e], cs[e], cs[e], cp[e]], np.zeros(21)]))
        assert np.allclose(ev, expect, atol=1e-6 * cp[e])


def test_abs_normal_jacobian_on_eigenvectors():
    """|A_n| v = |lambda| v on every eigenvector, |A_n|^2 = A_n^2, and the theta columns of
    both flux solvers are zero."""
    el, _, dt, att, _ = _case(4, 3, 12)
    _, _, normals, _ = scheme.geometry(el.jac)
    An, absAn = ve.abs_normal_jacobian(el.rho, el.lam, el.mu, att.ylam, att.ymu, att.omega, normals[:, 2])
    for e in range(4):
        w, V = np.linalg.eig(An[e])
        for k in range(27):
            v = V[:, k]
            lhs = absAn[e] @ v
            scale = np.abs(absAn[e]).max() * np.linalg.norm(v)
            assert np.linalg.norm(lhs - abs(w[k].real) * v) <= 1e-9 * scale
        # rows span many decades (stresses, velocities, anelastic functions): compare
        # each row against its own largest entry
        sq, A2 = absAn[e] @ absAn[e], An[e] @ An[e]
        row = np.abs(A2).max(axis=1, keepdims=True)
        assert (np.abs(sq - A2) <= 1e-7 * row).all()
    star, src, loc, nb = _setup(el, att)
    assert not loc[:, :, :, 9:].any() and not nb[:, :, :, 9:].any()


@pytest.mark.parametrize("order_n", [2, 4])
def test_without_source_elastic_part_is_the_elastic_step(order_n):
    """With the source switched off the nine elastic quantities evolve exactly as in the
    elastic oracle (the anelastic functions do not feed back), while the anelastic
    functions still change (they are driven by the velocity field)."""
    el, conn, dt, att, Q = _case(12, order_n, 13)
    star, src, loc, nb = _setup(el, att)
    q27, i27 = ve.ader_step(Q, star, np.zeros_like(src), loc, nb, conn.neighbours, conn.faces,
                            conn.orient, dt, order_n)
    s9, l9, n9 = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    q9, i9 = scheme.ader_step(Q[:, :, :9], s9, l9, n9, conn.neighbours, conn.faces, conn.orient,
                              dt, order_n)
    assert np.allclose(q27[:, :, :9], q9, rtol=0, atol=1e-12 * np.abs(q9).max())
    assert np.allclose(i27[:, :, :9], i9, rtol=0, atol=1e-12 * np.abs(i9).max())
    assert np.abs(q27[:, :, 9:] - Q[:, :, 9:]).max() > 1e-6 * np.abs(Q[:, :, 9:]).max()
    # with the source the elastic part differs
    q27s, _ = ve.ader_step(Q, star, src, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, order_n)
    assert np.abs(q27s[:, :, :6] - q9[:, :, :6]).max() > 1e-6 * np.abs(q9[:, :, :6] - Q[:, :, :6]).max()


def _relaxation_closed_form(q0, omega, t):
    """Solution of sigma_i' = -sum_l theta^l_i, theta^l' = -omega_l theta^l (velocities
    constant) at time t and its integral over [0, t]; q0 (..., 27), omega (3,)."""
    q = np.array(q0, dtype=np.float64, copy=True)
    integ = np.array(q0, dtype=np.float64, copy=True) * t
    for l in range(3):
        r0 = ve.theta_index(l, 0)
        th = q0[..., r0:r0 + 6]
        w = omega[l]
        decay = np.exp(-w * t)
        q[..., r0:r0 + 6] = th * decay
        integ[..., r0:r0 + 6] = th * (1 - decay) / w
        q[..., 0:6] -= th * (1 - decay) / w
        integ[..., 0:6] -= th * (t / w - (1 - decay) / w ** 2)
    return q, integ


@pytest.mark.parametrize("order_n", [1, 3, 6])
def test_pure_source_step_is_truncated_relaxation(order_n):
    """Star matrices and flux solvers zeroed: D^d = Q (E^T)^d, so the step is the Taylor
    polynomial of degree N+1 of the relaxation ODE's solution; it matches the closed form
    within the Taylor remainder (omega dt)^{N+2} / (N+2)! (times a safety factor)."""
    el, conn, dt, att, Q = _case(6, order_n, 14)
    star, src, loc, nb = _setup(el, att)
    z = np.zeros_like
    q, I = ve.ader_step(Q, z(star), src, z(loc), z(nb), conn.neighbours, conn.faces, conn.orient,
                        dt, order_n)
    for e in range(6):
        ref_q, ref_i = _relaxation_closed_form(Q[e], att.omega[e], dt)
        x = (att.omega[e] * dt).max()
        rem = 4.0 * x ** (order_n + 2) / factorial(order_n + 2)
        scale_q = np.abs(Q[e]).max()
        assert np.abs(q[e] - ref_q).max() <= rem * scale_q + 1e-13 * scale_q
        assert np.abs(I[e] - ref_i).max() <= rem * scale_q * dt + 1e-13 * scale_q * dt
    # and the update is not the identity (the source acts)
    assert np.abs(q - Q).max() > 1e-3 * np.abs(Q).max()


def test_constant_state_on_periodic_mesh_only_relaxes():
    """A spatially constant state on the periodic mesh with one material and one set of
    attenuation parameters: the volume term and the fluxes cancel, so each element follows
    the pure relaxation (the Taylor polynomial of degree N+1) and the higher basis
    coefficients stay zero."""
    N = 3
    mesh = wl.periodic_cube_mesh(3)
    el = mesh.elements
    E = el.rho.size
    dt = wl.cfl_time_step(el, N, cfl=0.3)
    omega = np.tile(np.array([0.01, 0.1, 0.4]) / dt, (E, 1))
    att = wl.Attenuation(omega, 0.02 * el.lam[:, None] * np.ones((1, 3)), 0.03 * el.mu[:, None] * np.ones((1, 3)))
    star, src, loc, nb = _setup(el, att)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(27)
    Q = np.zeros((E, basis.n_basis(N), 27))
    Q[:, 0, :] = c
    q, _ = ve.ader_step(Q, star, src, loc, nb, mesh.conn.neighbours, mesh.conn.faces,
                        mesh.conn.orient, dt, N)
    # the step's own relaxation polynomial: sum_{d <= N+1} c (dt E^T)^d / d!
    ET = src[0].T * dt
    poly = np.zeros((27, 27))
    term = np.eye(27)
    for d in range(N + 2):
        poly += term / factorial(d)
        term = term @ ET
    assert np.allclose(q[:, 0, :], (c @ poly)[None, :], rtol=0, atol=1e-11 * np.abs(c).max())
    assert np.abs(q[:, 1:, :]).max() <= 1e-11 * np.abs(c).max()


def test_linearity():
    el, conn, dt, att, Q = _case(10, 3, 15)
    star, src, loc, nb = _setup(el, att)
    a, _ = ve.ader_step(Q, star, src, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, 3)
    Q2 = wl.random_dofs_viscoelastic(10, basis.n_basis(3), el, att, seed=99)
    b, _ = ve.ader_step(Q2, star, src, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, 3)
    c, _ = ve.ader_step(2.5 * Q - Q2, star, src, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, 3)
    assert np.allclose(c, 2.5 * a - b, rtol=0, atol=1e-11 * np.abs(c).max())
