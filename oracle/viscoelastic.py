"""Direct FP64 evaluation of one ADER-DG step of the 27-quantity viscoelastic-shaped system
(oracle; test infrastructure).

The paper names viscoelastic attenuation with three mechanisms (27 quantities) as one of
SeisSol's rheologies (Sec. 5.1) but gives no equations for it.  Reading used here (the
common memory-variable form of a generalised Maxwell / standard linear solid body,
written for this oracle): q = (sxx, syy, szz, sxy, syz, sxz, u, v, w, theta^1, theta^2,
theta^3) with six anelastic functions theta^l per mechanism l = 1..3, and

    q_t + A q_x + B q_y + C q_z = E q,

* A, B, C (27 x 27): the elastic Jacobians in the leading 9 x 9 block; the rows of theta^l
  are omega_l times the stress-velocity block of the elastic Jacobian evaluated with the
  anelastic moduli (Y^lambda_l, Y^mu_l) in place of (lambda, mu); the columns of the
  theta quantities are zero (the anelastic functions have no flux);
* E (27 x 27), the reactive source: d sigma_i / dt gets -sum_l theta^l_i, and
  d theta^l_i / dt gets -omega_l theta^l_i.

The scheme of Sec. 5.1.1 extended by the source term (the source is local, so it enters
each equation through the time-integrated DOFs like the volume term does):

    D^{d+1}_kp = sum_x Ktilde^x_kl D^d_lq Astar^x_pq + D^d_kq E_pq,   D^0 = Q
    I_kp       = sum_{d=0}^{N} dt^{d+1}/(d+1)! D^d_kp
    Q_kp      += sum_x Khat^x_kl I_lq Astar^x_pq + I_kq E_pq
                 + sum_sigma (M^-1 F^-_sigma)_kl I_lq (Aloc_sigma)_pq
                 + sum_sigma (M^-1 F^+_{sigma,j,h})_kl I^nb_lq (Anb_sigma)_pq

with dense 27 x 27 per-element matrices (no block pattern exploited), the unfactorised
flux matrices of oracle/basis.py and the upwind flux solvers of the homogeneous material,
-(2|S|/|J|)(A_n +- |A_n|)/2, where A_n = n_x A + n_y B + n_z C (27 x 27).  A_n has the
spectrum {0, +-c_s, +-c_p} of the elastic block (plus zeros) and is diagonalisable, so
|A_n| follows from Sylvester's formula over those five values as in the elastic case.
The attenuation parameters are inputs (synthetic, see workload.attenuation); physics is
not pinned, the arithmetic is.
"""
from __future__ import annotations

import numpy as np

from . import basis
from . import scheme

N_MECH = 3
N_QUANTITIES = 9 + 6 * N_MECH      # 27


def theta_index(l, i):
    """Quantity index of component i (0..5) of the anelastic function of mechanism l."""
    return 9 + 6 * l + i


def jacobians(rho, lam, mu, ylam, ymu, omega):
    """A, B, C (each (E, 27, 27)).  ylam, ymu, omega: (E, 3) per mechanism."""
    rho, lam, mu = (np.asarray(v, dtype=np.float64) for v in (rho, lam, mu))
    ylam, ymu, omega = (np.asarray(v, dtype=np.float64) for v in (ylam, ymu, omega))
    E = rho.shape[0]
    el = scheme.elastic_jacobians(rho, lam, mu)
    out = []
    for d in range(3):
        J = np.zeros((E, N_QUANTITIES, N_QUANTITIES))
        J[:, :9, :9] = el[d]
        for l in range(N_MECH):
            an = scheme.elastic_jacobians(rho, ylam[:, l], ymu[:, l])[d]
            r0 = theta_index(l, 0)
            J[:, r0:r0 + 6, 6:9] = omega[:, l, None, None] * an[:, 0:6, 6:9]
        out.append(J)
    return tuple(out)


def source_matrix(omega):
    """E (E, 27, 27) of q_t + ... = E q."""
    omega = np.asarray(omega, dtype=np.float64)
    E = omega.shape[0]
    S = np.zeros((E, N_QUANTITIES, N_QUANTITIES))
    for l in range(N_MECH):
        for i in range(6):
            t = theta_index(l, i)
            S[:, i, t] = -1.0
            S[:, t, t] = -omega[:, l]
    return S


def star_matrices(rho, lam, mu, ylam, ymu, omega, jac):
    """Astar^x = sum_j (d xi_x / d x_j) A^j, shape (E, 3, 27, 27)."""
    jacs = np.stack(jacobians(rho, lam, mu, ylam, ymu, omega), axis=1)
    inv, _, _, _ = scheme.geometry(jac)
    return np.einsum('exj,ejpq->expq', inv, jacs)


def abs_normal_jacobian(rho, lam, mu, ylam, ymu, omega, normal):
    """(A_n, |A_n|) by Sylvester's formula over the distinct eigenvalues {0, +-cs, +-cp}."""
    A, Bm, C = jacobians(rho, lam, mu, ylam, ymu, omega)
    n = np.asarray(normal, dtype=np.float64)
    An = n[:, 0, None, None] * A + n[:, 1, None, None] * Bm + n[:, 2, None, None] * C
    cp = np.sqrt((lam + 2.0 * mu) / rho)
    cs = np.sqrt(mu / rho)
    eig = [np.zeros_like(cp), cp, -cp, cs, -cs]
    eye = np.broadcast_to(np.eye(N_QUANTITIES), An.shape)
    out = np.zeros_like(An)
    for i, li in enumerate(eig):
        term = np.abs(li)[:, None, None] * eye
        for j, lj in enumerate(eig):
            if i != j:
                term = np.matmul(term, (An - lj[:, None, None] * eye) / (li - lj)[:, None, None])
        out += term
    return An, out


def flux_solvers(rho, lam, mu, ylam, ymu, omega, jac):
    """(Aloc, Anb) each (E, 4, 27, 27)."""
    _, det, normals, areas = scheme.geometry(jac)
    E = det.shape[0]
    loc = np.zeros((E, 4, N_QUANTITIES, N_QUANTITIES))
    nb = np.zeros_like(loc)
    for s in range(4):
        An, absAn = abs_normal_jacobian(rho, lam, mu, ylam, ymu, omega, normals[:, s])
        scale = -(2.0 * areas[:, s] / np.abs(det))[:, None, None]
        loc[:, s] = scale * 0.5 * (An + absAn)
        nb[:, s] = scale * 0.5 * (An - absAn)
    return loc, nb


def setup_element_matrices(rho, lam, mu, ylam, ymu, omega, jac):
    """Star matrices, source matrices and flux solvers of every element (FP64)."""
    star = star_matrices(rho, lam, mu, ylam, ymu, omega, jac)
    src = source_matrix(omega)
    loc, nb = flux_solvers(rho, lam, mu, ylam, ymu, omega, jac)
    return star, src, loc, nb


def derivatives_and_time_integral(Q, star, src, dt, order_n):
    """D^0..D^N and I with the source term (the CK recursion above)."""
    m = basis.float_matrices(order_n)
    coeff = scheme.time_integral_coefficients(dt, order_n)
    D = [np.asarray(Q, dtype=np.float64)]
    for _ in range(order_n):
        nxt = sum(np.matmul(np.matmul(m['Ktilde'][x], D[-1]), np.swapaxes(star[:, x], -1, -2))
                  for x in range(3))
        nxt = nxt + np.matmul(D[-1], np.swapaxes(src, -1, -2))
        D.append(nxt)
    I = sum(coeff[d] * D[d] for d in range(order_n + 1))
    return D, I


def local_update(Q, I, star, src, flux_loc, order_n):
    """Q + volume + source + local flux."""
    out = scheme.local_update(Q, I, star, flux_loc, order_n)
    return out + np.matmul(I, np.swapaxes(src, -1, -2))


def ader_step(Q, star, src, flux_loc, flux_nb, neighbours, faces, orient, dt, order_n,
              with_neighbours=True):
    """One step; Q (E, B, 27) [element, basis, quantity]; returns (Q_new, I)."""
    _, I = derivatives_and_time_integral(Q, star, src, dt, order_n)
    Qn = local_update(Q, I, star, src, flux_loc, order_n)
    if with_neighbours:
        Qn = scheme.neighbour_update(Qn, I, flux_nb, neighbours, faces, orient, order_n)
    return Qn, I
