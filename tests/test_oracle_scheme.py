"""Pins of the oracle's scheme: Jacobians, geometry, flux solvers, the CK recursion and
the whole step against the elastic plane wave (observed order = O, Sec. 5)."""
import numpy as np
import pytest

import workload as wl
from oracle import basis, planewave, scheme


def test_jacobian_eigenstructure():
    rho, lam, mu = 2500.0, 3e10, 2e10
    rng = np.random.default_rng(3)
    for _ in range(5):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        A, B, C = scheme.elastic_jacobians(rho, lam, mu)
        An = n[0] * A + n[1] * B + n[2] * C
        cp, cs = np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)
        ev = np.sort(np.linalg.eigvals(An).real)
        assert np.allclose(ev, np.sort([-cp, -cs, -cs, 0, 0, 0, cs, cs, cp]), atol=1e-6 * cp)
        r, c = planewave.p_wave_vector(rho, lam, mu, n)
        assert np.allclose(An @ r, c * r, rtol=1e-13, atol=1e-13 * np.abs(c * r).max())


def test_abs_normal_jacobian_against_eigendecomposition():
    """Compared in impedance-scaled units (stress rows / columns divided by rho c_p), where
    every block of A_n has the scale of a wave speed."""
    rng = np.random.default_rng(4)
    rho, lam, mu = 2200.0, 1.5e10, 3.5e10
    cp = np.sqrt((lam + 2 * mu) / rho)
    Dg = np.diag([1.0 / (rho * cp)] * 6 + [1.0] * 3)
    Di = np.linalg.inv(Dg)
    for _ in range(4):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        An, absAn = scheme.abs_normal_jacobian(rho, lam, mu, n)
        w, V = np.linalg.eig(An)
        ref = (V @ np.diag(np.abs(w)) @ np.linalg.inv(V)).real
        As, absAs, refs = Dg @ An @ Di, Dg @ absAn @ Di, Dg @ ref @ Di
        assert np.allclose(absAs, refs, atol=1e-9 * cp)
        assert np.allclose(absAs @ absAs, As @ As, atol=1e-12 * cp * cp)
        assert np.allclose(absAs @ As, As @ absAs, atol=1e-12 * cp * cp)


def test_geometry_against_cross_products():
    el = wl.random_elements(50, seed=5)
    inv, det, normals, areas = scheme.geometry(el.jac)
    ref = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    X = np.einsum('eij,vj->evi', el.jac, ref)
    closed = np.zeros((50, 3))
    for s, (a, b, c) in enumerate(basis.FACE_VERTICES):
        cr = np.cross(X[:, b] - X[:, a], X[:, c] - X[:, a])
        assert np.allclose(areas[:, s], 0.5 * np.linalg.norm(cr, axis=1), rtol=1e-13)
        assert np.allclose(normals[:, s], cr / np.linalg.norm(cr, axis=1)[:, None], atol=1e-13)
        closed += areas[:, s, None] * normals[:, s]
    assert np.abs(closed).max() < 1e-12                  # closed surface
    assert np.allclose(det, np.linalg.det(el.jac))


def test_star_identity_geometry():
    jac = np.eye(3)[None].repeat(2, 0)
    star = scheme.star_matrices(np.array([2000.0, 2500.0]), np.array([1e10, 2e10]),
                                np.array([3e10, 1e10]), jac)
    A, B, C = scheme.elastic_jacobians(np.array([2000.0, 2500.0]), np.array([1e10, 2e10]),
                                       np.array([3e10, 1e10]))
    assert np.array_equal(star[:, 0], A) and np.array_equal(star[:, 1], B)
    assert np.array_equal(star[:, 2], C)
    assert all(int((np.abs(star[0, d]) > 0).sum()) == 8 for d in range(3))


def test_flux_split():
    el = wl.random_elements(10, seed=6)
    loc, nb = scheme.flux_solvers(el.rho, el.lam, el.mu, el.jac)
    _, det, normals, areas = scheme.geometry(el.jac)
    for s in range(4):
        A, B, C = scheme.elastic_jacobians(el.rho, el.lam, el.mu)
        n = normals[:, s]
        An = n[:, 0, None, None] * A + n[:, 1, None, None] * B + n[:, 2, None, None] * C
        scale = -(2 * areas[:, s] / det)[:, None, None]
        assert np.allclose(loc[:, s] + nb[:, s], scale * An, rtol=1e-12,
                           atol=1e-12 * np.abs(scale * An).max())
        # A_n^+ has eigenvalues >= 0, A_n^- <= 0 (upwind split)
        evp = np.linalg.eigvals(loc[0, s] / scale[0]).real
        evm = np.linalg.eigvals(nb[0, s] / scale[0]).real
        tol = 1e-6 * np.abs(evp).max()
        assert evp.min() > -tol and evm.max() < tol


def test_time_integral_coefficients():
    c = scheme.time_integral_coefficients(0.1, 3)
    assert np.allclose(c, [0.1, 0.01 / 2, 0.001 / 6, 0.0001 / 24], rtol=1e-15)


def test_ck_derivative_of_linear_field():
    """For q linear in x, dq/dt = -sum_j A^j dq/dx_j is constant: D^1 holds exactly that
    constant (coefficient of phi_0) and D^2 = 0 (Eq. seissol:derivative)."""
    N = 3
    el = wl.random_elements(4, seed=7)
    rng = np.random.default_rng(8)
    a = rng.standard_normal(9)
    G = rng.standard_normal((9, 3))              # dq_p / dx_j
    pts, wts = planewave.tet_quadrature(6)
    phi = basis.evaluate_tet_basis(N, pts)
    Mdiag = np.array([float(basis.exact_matrices(N)['M'][i, i]) for i in range(phi.shape[1])])
    x = np.einsum('eij,qj->eqi', el.jac, pts)
    q = a[None, None] + np.einsum('pj,eqj->eqp', G, x)
    Q = np.einsum('qk,q,eqp->ekp', phi, wts, q) / Mdiag[None, :, None]
    star = scheme.star_matrices(el.rho, el.lam, el.mu, el.jac)
    D, _ = scheme.derivatives_and_time_integral(Q, star, 0.0, N)
    A, B, C = scheme.elastic_jacobians(el.rho, el.lam, el.mu)
    qt = -(np.einsum('epq,q->ep', A, G[:, 0]) + np.einsum('epq,q->ep', B, G[:, 1])
           + np.einsum('epq,q->ep', C, G[:, 2]))
    scale = np.abs(qt).max()
    assert np.allclose(D[1][:, 0], qt, atol=1e-11 * scale)
    assert np.abs(D[1][:, 1:]).max() < 1e-11 * scale
    assert np.abs(D[2]).max() < 1e-11 * scale * np.abs(star).max()


def test_step_is_linear():
    N = 2
    E = 16
    el = wl.random_elements(E, seed=9)
    conn = wl.random_connectivity(E, seed=10)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    Q = wl.random_dofs(E, basis.n_basis(N), seed=11)
    dt = wl.cfl_time_step(el, N)
    q1, i1 = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, N)
    q2, i2 = scheme.ader_step(3.0 * Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, N)
    assert np.allclose(q2, 3.0 * q1, rtol=1e-13, atol=1e-13 * np.abs(q1).max())


def test_constant_state_is_preserved():
    mesh = wl.periodic_cube_mesh(3)
    el = mesh.elements
    N = 2
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    Q = np.zeros((el.rho.size, basis.n_basis(N), 9))
    Q[:, 0, :] = np.arange(1, 10)
    dt = wl.cfl_time_step(el, N)
    q1, _ = scheme.ader_step(Q, star, loc, nb, mesh.conn.neighbours, mesh.conn.faces,
                             mesh.conn.orient, dt, N)
    assert np.abs(q1 - Q).max() < 1e-12 * np.abs(Q).max()


@pytest.mark.parametrize("N", [1, 2, 3])
def test_plane_wave_convergence(N):
    """Observed L2 convergence order matches O = N + 1 (Sec. 5, plane-wave validation)."""
    k = 2 * np.pi * np.array([1.0, 1.0, 0.0])
    T = 0.05
    errs = []
    for n in (3, 6):
        mesh = wl.periodic_cube_mesh(n)
        el = mesh.elements
        star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
        steps = int(np.ceil(T / wl.cfl_time_step(el, N, cfl=0.3)))
        dt = T / steps
        Q = planewave.project(mesh, N, 0.0, k, 1.0, 2.0, 1.0)
        for _ in range(steps):
            Q, _ = scheme.ader_step(Q, star, loc, nb, mesh.conn.neighbours, mesh.conn.faces,
                                    mesh.conn.orient, dt, N)
        errs.append(planewave.l2_error(mesh, N, Q, T, k, 1.0, 2.0, 1.0))
    rate = np.log2(errs[0] / errs[1])
    # velocities u, v and normal stresses; observed order close to N + 1
    assert rate[6] > N + 1 - 0.35 and rate[0] > N + 1 - 0.35, rate
