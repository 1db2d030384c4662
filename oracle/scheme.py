"""Direct FP64 evaluation of one ADER-DG step on tetrahedra (oracle; test infrastructure).

Follows Sec. 5.1.1 of the paper:
  Eq. seissol:derivative   D^{d+1}_kp = sum_x Ktilde^x_kl D^d_lq Astar^x_pq,  D^0 = Q
  Eq. seissol:timeint      I_kp = sum_{d=0}^{N} dt^{d+1}/(d+1)! D^d_kp
  Eq. seissol:correction_local
                           Q_kp += sum_x Khat^x_kl I_lq Astar^x_pq
                                   + sum_sigma (M^-1 F^-_sigma)_kl I_lq (Aloc_sigma)_pq
  Eq. seissol:correction_neigh
                           Q_kp += sum_sigma (M^-1 F^+_{sigma,j,h})_kl I^{nb}_lq (Anb_sigma)_pq
with unfactorised dense B x B flux matrices, dense Ktilde / Khat, no equivalent sparsity
patterns and no reordering (the plain definition).  The third volume term uses C* (the
paper prints B*, a typo).  Matrix products of two operands at a time are evaluated with
numpy's matmul.

The pieces the paper leaves out are the standard velocity-stress elastic system
(q = sxx, syy, szz, sxy, syz, sxz, u, v, w), star matrices
Astar^x = sum_j (d xi_x / d x_j) A^j (element-dependent linear combinations of the
Jacobians, Sec. 5.1.1), and the upwind (Godunov) flux of a homogeneous material,
    Aloc_sigma = -(2 |S_sigma| / |J|) (A_n + |A_n|) / 2,
    Anb_sigma  = -(2 |S_sigma| / |J|) (A_n - |A_n|) / 2,
A_n = n_x A + n_y B + n_z C with the outward unit normal n, face area |S| and Jacobian
determinant |J| (the factor 2 is the inverse area of the reference triangle).  |A_n| is
evaluated with Sylvester's formula over the five distinct eigenvalues 0, +-c_s, +-c_p.
"""
from __future__ import annotations

from math import factorial

import numpy as np

from . import basis

N_QUANTITIES = 9

# reference outward unit normals and areas of faces 1..4 (face vertex lists in basis.py)
_REF_NORMALS = np.array([[0.0, 0.0, -1.0], [0.0, -1.0, 0.0], [-1.0, 0.0, 0.0],
                         [1.0, 1.0, 1.0]])
_REF_NORMALS[3] /= np.sqrt(3.0)
_REF_AREAS = np.array([0.5, 0.5, 0.5, np.sqrt(3.0) / 2.0])


def elastic_jacobians(rho, lam, mu):
    """A, B, C (each (..., 9, 9)) of q_t + A q_x + B q_y + C q_z = 0 (Eq. linearpde) for
    isotropic elasticity in velocity-stress form."""
    rho, lam, mu = (np.asarray(v, dtype=np.float64) for v in (rho, lam, mu))
    shape = rho.shape + (9, 9)
    A = np.zeros(shape)
    Bm = np.zeros(shape)
    C = np.zeros(shape)
    l2m = lam + 2.0 * mu
    ir = 1.0 / rho
    # x direction
    A[..., 0, 6] = -l2m
    A[..., 1, 6] = -lam
    A[..., 2, 6] = -lam
    A[..., 3, 7] = -mu
    A[..., 5, 8] = -mu
    A[..., 6, 0] = -ir
    A[..., 7, 3] = -ir
    A[..., 8, 5] = -ir
    # y direction
    Bm[..., 0, 7] = -lam
    Bm[..., 1, 7] = -l2m
    Bm[..., 2, 7] = -lam
    Bm[..., 3, 6] = -mu
    Bm[..., 4, 8] = -mu
    Bm[..., 6, 3] = -ir
    Bm[..., 7, 1] = -ir
    Bm[..., 8, 4] = -ir
    # z direction
    C[..., 0, 8] = -lam
    C[..., 1, 8] = -lam
    C[..., 2, 8] = -l2m
    C[..., 4, 7] = -mu
    C[..., 5, 6] = -mu
    C[..., 6, 5] = -ir
    C[..., 7, 4] = -ir
    C[..., 8, 2] = -ir
    return A, Bm, C


def geometry(jac):
    """Per element (E,3,3) Jacobian dx/dxi -> (inverse (E,3,3), det (E,), outward unit
    normals (E,4,3), face areas (E,4)).  Normals use the covariant transform J^-T n_ref;
    areas use |S| = |J| |J^-T n_ref| |S_ref|."""
    jac = np.asarray(jac, dtype=np.float64)
    inv = np.linalg.inv(jac)
    det = np.linalg.det(jac)
    cov = np.einsum('eji,sj->esi', inv, _REF_NORMALS)      # J^-T n_ref
    norm = np.linalg.norm(cov, axis=-1)
    normals = cov / norm[..., None]
    areas = np.abs(det)[:, None] * norm * _REF_AREAS[None, :]
    return inv, det, normals, areas


def star_matrices(rho, lam, mu, jac):
    """Astar^x_pq = sum_j (d xi_x / d x_j) A^j_pq, shape (E, 3, 9, 9)."""
    A, Bm, C = elastic_jacobians(rho, lam, mu)
    inv, _, _, _ = geometry(jac)
    jacs = np.stack([A, Bm, C], axis=1)                      # (E, 3[j], 9, 9)
    return np.einsum('exj,ejpq->expq', inv, jacs)


def abs_normal_jacobian(rho, lam, mu, normal):
    """|A_n| by Sylvester's formula f(A) = sum_i f(l_i) prod_{j!=i} (A - l_j)/(l_i - l_j)
    over the distinct eigenvalues {0, +-cs, +-cp} of the diagonalisable A_n."""
    A, Bm, C = elastic_jacobians(rho, lam, mu)
    n = np.asarray(normal, dtype=np.float64)
    An = n[..., 0, None, None] * A + n[..., 1, None, None] * Bm + n[..., 2, None, None] * C
    cp = np.sqrt((lam + 2.0 * mu) / rho)
    cs = np.sqrt(mu / rho)
    eig = [np.zeros_like(cp), cp, -cp, cs, -cs]
    eye = np.broadcast_to(np.eye(9), An.shape)
    out = np.zeros_like(An)
    for i, li in enumerate(eig):
        term = np.abs(li)[..., None, None] * eye
        for j, lj in enumerate(eig):
            if i == j:
                continue
            term = np.matmul(term, (An - lj[..., None, None] * eye) / (li - lj)[..., None, None])
        out += term
    return An, out


def flux_solvers(rho, lam, mu, jac):
    """(Aloc, Anb) each (E, 4, 9, 9): upwind flux solvers of the four faces."""
    _, det, normals, areas = geometry(jac)
    E = det.shape[0]
    loc = np.zeros((E, 4, 9, 9))
    nb = np.zeros((E, 4, 9, 9))
    for s in range(4):
        An, absAn = abs_normal_jacobian(rho, lam, mu, normals[:, s])
        scale = -(2.0 * areas[:, s] / np.abs(det))[:, None, None]
        loc[:, s] = scale * 0.5 * (An + absAn)
        nb[:, s] = scale * 0.5 * (An - absAn)
    return loc, nb


def time_integral_coefficients(dt, order_n):
    """dt^{d+1} / (d+1)!, d = 0..N (Eq. seissol:timeint)."""
    return np.array([dt ** (d + 1) / factorial(d + 1) for d in range(order_n + 1)])


def _apply(Kmat, X, Astar):
    """K_kl X_elq A_epq -> (E, B, 9) for a global K and per-element A."""
    return np.matmul(np.matmul(Kmat, X), np.swapaxes(Astar, -1, -2))


def derivatives_and_time_integral(Q, star, dt, order_n):
    """D^0..D^N (list) and I, Eqs. seissol:derivative and seissol:timeint."""
    m = basis.float_matrices(order_n)
    coeff = time_integral_coefficients(dt, order_n)
    D = [np.asarray(Q, dtype=np.float64)]
    for _ in range(order_n):
        nxt = sum(_apply(m['Ktilde'][x], D[-1], star[:, x]) for x in range(3))
        D.append(nxt)
    I = sum(coeff[d] * D[d] for d in range(order_n + 1))
    return D, I


def local_update(Q, I, star, flux_loc, order_n):
    """Q + volume + local flux (Eq. seissol:correction_local)."""
    m = basis.float_matrices(order_n)
    out = np.array(Q, dtype=np.float64, copy=True)
    for x in range(3):
        out += _apply(m['Khat'][x], I, star[:, x])
    for s in range(4):
        out += _apply(m['FmHat'][s], I, flux_loc[:, s])
    return out


def neighbour_update(Q, I, flux_nb, neighbours, faces, orient, order_n, chunk=4096):
    """Q + neighbour flux (Eq. seissol:correction_neigh) with the 48 dense F^+."""
    m = basis.float_matrices(order_n)
    FpHat = m['FpHat']
    out = np.array(Q, dtype=np.float64, copy=True)
    E = Q.shape[0]
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        for s in range(4):
            nb = neighbours[e0:e1, s]
            F = FpHat[s, faces[e0:e1, s], orient[e0:e1, s]]          # (n, B, B)
            out[e0:e1] += np.matmul(np.matmul(F, I[nb]), np.swapaxes(flux_nb[e0:e1, s], -1, -2))
    return out


def ader_step(Q, star, flux_loc, flux_nb, neighbours, faces, orient, dt, order_n,
              with_neighbours=True):
    """One ADER-DG step.  Q (E, B, 9) indexed [element, basis k, quantity p]; returns
    (Q_new, I).  neighbours/faces/orient (E, 4) give Neigh, Face (= j) and Rot (= h)."""
    _, I = derivatives_and_time_integral(Q, star, dt, order_n)
    Qn = local_update(Q, I, star, flux_loc, order_n)
    if with_neighbours:
        Qn = neighbour_update(Qn, I, flux_nb, neighbours, faces, orient, order_n)
    return Qn, I


def setup_element_matrices(rho, lam, mu, jac):
    """Star matrices and flux solvers of every element (setup step, FP64)."""
    star = star_matrices(rho, lam, mu, jac)
    loc, nb = flux_solvers(rho, lam, mu, jac)
    return star, loc, nb


def ader_step_mixed(Q_list, orders_n, star, flux_loc, flux_nb, neighbours, faces, orient, dt):
    """One step of a p-adaptive mesh: element e has degree orders_n[e] and DOFs Q_list[e]
    (B_e x 9).  The local part is the plain step of degree N_e; the neighbour flux of
    face s couples B_e test functions with the neighbour's B_nb basis functions through
    M^-1 F^+ cropped to [B_e, B_nb] (the basis is hierarchical: the first C(n+3,3)
    functions of any degree span P_n, so the cropped matrix is exactly the integral of
    the two elements' own functions).  Returns (list of Q_new, list of I)."""
    E = len(Q_list)
    I_list = [None] * E
    out = [None] * E
    Nmax = int(max(orders_n))
    m = basis.float_matrices(Nmax)
    for e in range(E):
        N = int(orders_n[e])
        Q = np.asarray(Q_list[e], dtype=np.float64)[None]
        _, I = derivatives_and_time_integral(Q, star[e:e + 1], dt, N)
        I_list[e] = I[0]
        out[e] = local_update(Q, I, star[e:e + 1], flux_loc[e:e + 1], N)[0]
    for e in range(E):
        Be = basis.n_basis(int(orders_n[e]))
        for s in range(4):
            nb = int(neighbours[e, s])
            Bn = basis.n_basis(int(orders_n[nb]))
            F = m['FpHat'][s, faces[e, s], orient[e, s]][:Be, :Bn]
            out[e] = out[e] + F @ I_list[nb] @ flux_nb[e, s].T
    return out, I_list
