"""Elastic plane wave: closed form, L2 projection and L2 error (oracle; test infrastructure).

The paper validates both codes with a plane-wave problem and checks that the observed
convergence order matches the theoretical order O = N + 1 (Sec. 5, opening paragraph).
For a homogeneous isotropic medium and a wave vector k, n = k/|k|, the P wave
    q(x, t) = r sin(k.x - c_p |k| t),  r_v = n,  r_sigma = -(lambda I + 2 mu n n^T) / c_p
solves q_t + A q_x + B q_y + C q_z = 0 exactly (A_n r = c_p r).
"""
from __future__ import annotations

import numpy as np

from . import basis


def p_wave_vector(rho, lam, mu, normal):
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    cp = np.sqrt((lam + 2 * mu) / rho)
    S = -(lam * np.eye(3) + 2 * mu * np.outer(n, n)) / cp
    # quantity order: sxx, syy, szz, sxy, syz, sxz, u, v, w
    r = np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[1, 2], S[0, 2], n[0], n[1], n[2]])
    return r, cp


def exact(x, t, k, rho, lam, mu):
    """q at points x (..., 3) and time t -> (..., 9)."""
    k = np.asarray(k, dtype=np.float64)
    r, cp = p_wave_vector(rho, lam, mu, k)
    phase = x @ k - cp * np.linalg.norm(k) * t
    return np.sin(phase)[..., None] * r


def tet_quadrature(n_points: int = 10):
    """Collapsed (Duffy) Gauss-Legendre rule on the reference tetrahedron: points (n^3, 3)
    and weights; exact for polynomials of degree <= 2n - 3."""
    g, w = np.polynomial.legendre.leggauss(n_points)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    a, b, c = np.meshgrid(g, g, g, indexing='ij')
    wa, wb, wc = np.meshgrid(w, w, w, indexing='ij')
    zeta = c
    eta = b * (1 - c)
    xi = a * (1 - b) * (1 - c)
    weight = wa * wb * wc * (1 - b) * (1 - c) ** 2
    pts = np.stack([xi.ravel(), eta.ravel(), zeta.ravel()], axis=1)
    return pts, weight.ravel()


def project(mesh, order_n, t, k, rho, lam, mu, n_points=10):
    """L2 projection of the plane wave at time t onto every element: Q (E, B, 9)."""
    pts, wts = tet_quadrature(n_points)
    phi = basis.evaluate_tet_basis(order_n, pts)             # (nq, B)
    Mdiag = np.array([float(basis.exact_matrices(order_n)['M'][i, i])
                      for i in range(phi.shape[1])])
    x = mesh.vertices[:, 0][:, None, :] + np.einsum('eij,qj->eqi', mesh.elements.jac, pts)
    q = exact(x, t, k, rho, lam, mu)                          # (E, nq, 9)
    return np.einsum('qk,q,eqp->ekp', phi, wts, q) / Mdiag[None, :, None]


def l2_error(mesh, order_n, Q, t, k, rho, lam, mu, n_points=10):
    """Per-quantity L2 error of the DG solution Q against the plane wave at time t."""
    pts, wts = tet_quadrature(n_points)
    phi = basis.evaluate_tet_basis(order_n, pts)
    x = mesh.vertices[:, 0][:, None, :] + np.einsum('eij,qj->eqi', mesh.elements.jac, pts)
    q = exact(x, t, k, rho, lam, mu)
    qh = np.einsum('qk,ekp->eqp', phi, Q)
    det = np.abs(np.linalg.det(mesh.elements.jac))
    err2 = np.einsum('eqp,q,e->p', (qh - q) ** 2, wts, det)
    return np.sqrt(err2)
