"""Pins of the oracle's global matrices (exact rational identities and closed forms)."""
from fractions import Fraction
from math import comb

import numpy as np
import pytest
from scipy.special import eval_jacobi

from oracle import basis

ORDERS = [1, 2, 3, 4, 5]


def test_sizes():
    # B = C(N+3,3), Btilde = C(N+2,2): 10/20/35/56/84 and 6/10/15/21/28 (Sec. 5.1)
    assert [basis.n_basis(n) for n in range(2, 7)] == [10, 20, 35, 56, 84]
    assert [basis.n_face_basis(n) for n in range(2, 7)] == [6, 10, 15, 21, 28]


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("alpha", [0, 1, 4])
def test_jacobi_coefficients_match_library(n, alpha):
    c = basis.jacobi_coefficients(n, alpha)
    x = np.linspace(-1, 1, 7)
    mine = sum(float(ci) * x ** i for i, ci in enumerate(c))
    assert np.allclose(mine, eval_jacobi(n, alpha, 0, x), rtol=1e-13, atol=1e-13)


def test_basis_values_match_collapsed_formula():
    # evaluate phi_pqr from its collapsed-coordinate definition with scipy's Jacobi
    N = 4
    rng = np.random.default_rng(0)
    pts = rng.dirichlet([1, 1, 1, 1], 20)[:, :3]
    mine = basis.evaluate_tet_basis(N, pts)
    xi, eta, zeta = pts.T
    s1, s2 = 1 - eta - zeta, 1 - zeta
    for k, (p, q, r) in enumerate(basis.tet_indices(N)):
        ref = (eval_jacobi(p, 0, 0, 2 * xi / s1 - 1) * s1 ** p
               * eval_jacobi(q, 2 * p + 1, 0, 2 * eta / s2 - 1) * s2 ** q
               * eval_jacobi(r, 2 * p + 2 * q + 2, 0, 2 * zeta - 1))
        assert np.allclose(mine[:, k], ref, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("N", ORDERS)
def test_mass_matrix_diagonal_and_volume(N):
    M = basis.exact_matrices(N)["M"]
    B = M.shape[0]
    assert M[0, 0] == Fraction(1, 6)          # phi_0 = 1, |T| = 1/6
    for i in range(B):
        assert M[i, i] > 0
        for j in range(B):
            if i != j:
                assert M[i, j] == 0


@pytest.mark.parametrize("N", ORDERS)
def test_face_basis_orthogonal(N):
    W = basis.exact_matrices(N)["W"]
    assert W[0] == Fraction(1, 2)             # psi_0 = 1, |triangle| = 1/2


@pytest.mark.parametrize("N", ORDERS)
def test_integration_by_parts(N):
    """K^d + K^dT = int_dT phi_k phi_l n_d dS.  The face integral is 2|S_ref| F^-_sigma
    n_ref,d: face 4 contributes +F^-_4 for every d; the coordinate face with normal -e_d
    (face 3 for xi, 2 for eta, 1 for zeta) contributes -F^-."""
    ex = basis.exact_matrices(N)
    K, Fm = ex["K"], ex["Fm"]
    minus_face = {0: 2, 1: 1, 2: 0}
    for d in range(3):
        lhs = K[d] + K[d].T
        rhs = Fm[3] - Fm[minus_face[d]]
        assert (lhs == rhs).all()


@pytest.mark.parametrize("N", ORDERS)
def test_derivative_staircase(N):
    """Ktilde_kl != 0 only if deg(phi_k) < deg(phi_l), so D^delta has C(N-delta+3,3)
    non-zero rows (Sec. 5.1.2)."""
    ex = basis.exact_matrices(N)
    deg = [sum(t) for t in basis.tet_indices(N)]
    for d in range(3):
        Kt = ex["Ktilde"][d]
        for k in range(Kt.shape[0]):
            for l in range(Kt.shape[1]):
                if Kt[k, l] != 0:
                    assert deg[k] < deg[l]
    # Khat has only C(N+2,3) non-zero columns (l of degree < N)
    Kh = basis.float_matrices(N)["Khat"]
    nzcols = np.nonzero(np.abs(Kh).sum(axis=(0, 1)))[0]
    assert nzcols.max() + 1 == comb(N + 2, 3)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_flux_factorisation_exact(N):
    """M^-1 F^- = Rhat R^T and M^-1 F^+_{s,j,h} = Rhat^s f^h R^jT exactly (Eqs.
    seissol:correction_local and seissol:correction_neigh)."""
    ex = basis.exact_matrices(N)
    for s in range(4):
        assert (ex["Rhat"][s].dot(ex["R"][s].T) == ex["FmHat"][s]).all()
        for j in range(4):
            for h in range(3):
                prod = ex["Rhat"][s].dot(ex["f"][h]).dot(ex["R"][j].T)
                assert (prod == ex["FpHat"][s, j, h]).all()


@pytest.mark.parametrize("N", [2, 3])
def test_neighbour_flux_symmetry(N):
    """Theta_h is a measure-preserving involution, so F^+_{s,j,h} = (F^+_{j,s,h})^T; and
    phi_0 = 1 makes column 0 of every F^+_{s,.,.} equal to column 0 of F^-_s."""
    ex = basis.exact_matrices(N)
    for s in range(4):
        for j in range(4):
            for h in range(3):
                assert (ex["Fp"][s, j, h] == ex["Fp"][j, s, h].T).all()
                assert (ex["Fp"][s, j, h][:, 0] == ex["Fm"][s][:, 0]).all()


def test_face_mass_rank():
    # F^-_sigma is the Gram matrix of the traces: rank = Btilde (traces span P_N(face))
    N = 3
    Fm = basis.float_matrices(N)["Fm"]
    for s in range(4):
        assert np.linalg.matrix_rank(Fm[s], tol=1e-10) == basis.n_face_basis(N)


def test_known_sparsity_counts():
    # stiffness non-zeros at order 6 (N = 5): 294 / 672 / 742 of 3136
    K = basis.float_matrices(5)["K"]
    assert [int((np.abs(K[d]) > 0).sum()) for d in range(3)] == [294, 672, 742]
