"""Exact global matrices of the tetrahedral ADER-DG scheme (oracle; test infrastructure).

Everything here is computed in exact rational arithmetic (Python integers / Fractions)
and rounded to float64 only at the very end, so the oracle's global matrices are the
correctly rounded values of their definitions.

Definitions (Sec. 5.1 and Sec. 3 of the paper; readings where the paper is silent):

* Reference tetrahedron T = {xi, eta, zeta >= 0, xi + eta + zeta <= 1}.
* Basis: Dubiner's orthogonal polynomials (Sec. 5.1 names them, without formula)
      phi_{pqr} = P_p^{(0,0)}(2 xi / s1 - 1) s1^p * P_q^{(2p+1,0)}(2 eta / s2 - 1) s2^q
                  * P_r^{(2p+2q+2,0)}(2 zeta - 1),   s1 = 1 - eta - zeta, s2 = 1 - zeta,
  unnormalised, ordered by total degree d = p+q+r, then lexicographically in (p, q).
  The first C(n+3,3) functions span the polynomials of degree <= n.
* Face basis on the reference triangle {chi1, chi2 >= 0, chi1 + chi2 <= 1}:
      psi_{pq} = P_p^{(0,0)}(2 chi1 / (1 - chi2) - 1) (1 - chi2)^p P_q^{(2p+1,0)}(2 chi2 - 1),
  ordered by degree, then p.
* M_kl = int_T phi_k phi_l,   K^d_kl = int_T (d phi_k / d xi_d) phi_l   (Eq. stiffnesskernel
  convention), Khat^d = M^-1 K^d,   Ktilde^d = -M^-1 (K^d)^T.
* Faces: 1: zeta=0 (V0,V2,V1), 2: eta=0 (V0,V1,V3), 3: xi=0 (V0,V3,V2), 4: xi+eta+zeta=1
  (V1,V2,V3), with V0=(0,0,0), V1=(1,0,0), V2=(0,1,0), V3=(0,0,1); face sigma is
  parametrised as X_sigma(chi) = Va + chi1 (Vb - Va) + chi2 (Vc - Va), which makes the
  right-hand normal (Vb-Va) x (Vc-Va) point outwards.
* Neighbour orientation h in {0,1,2}: the neighbour's parameter of the point chi of the
  local face is Theta_h(chi) = (chi2, chi1), (1-chi1-chi2, chi2), (chi1, 1-chi1-chi2).
* F^-_sigma,kl = int_tri phi_k(X_sigma(chi)) phi_l(X_sigma(chi)) dchi,
  F^+_{sigma,j,h},kl = int_tri phi_k(X_sigma(chi)) phi_l(X_j(Theta_h(chi))) dchi
  (unfactorised flux matrices; Eq. seissol:correction_local / correction_neigh), and the
  factorisation R^sigma_lm = <phi_l o X_sigma, psi_m> / <psi_m, psi_m>,
  f^h_mn = <psi_n o Theta_h, psi_m> / <psi_m, psi_m>, W = diag <psi_m, psi_m>,
  Rhat^sigma = M^-1 R^sigma W, so that M^-1 F^- = Rhat R^T and M^-1 F^+ = Rhat f^h R^jT.

Integrals of monomials are exact:  int_T xi^a eta^b zeta^c = a! b! c! / (a+b+c+3)!,
int_tri chi1^a chi2^b = a! b! / (a+b+2)!  (Dirichlet integrals).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb, factorial, lcm

import numpy as np

TET_VERTICES = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))
FACE_VERTICES = ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3))


def n_basis(order_n: int) -> int:
    """B = C(N+3, 3) for polynomial degree N (Sec. 5.1)."""
    return comb(order_n + 3, 3)


def n_face_basis(order_n: int) -> int:
    """Btilde = C(N+2, 2) (Sec. 5.1.1)."""
    return comb(order_n + 2, 2)


# --------------------------------------------------------------------------- polynomials
# A polynomial is a dict {exponent tuple: Fraction}.

def _padd(a, b):
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, 0) + v
    return {k: v for k, v in out.items() if v != 0}


def _pmul(a, b):
    out = {}
    for ka, va in a.items():
        for kb, vb in b.items():
            k = tuple(x + y for x, y in zip(ka, kb))
            out[k] = out.get(k, 0) + va * vb
    return {k: v for k, v in out.items() if v != 0}


def _pscale(a, s):
    return {k: v * s for k, v in a.items() if v * s != 0}


def _ppow(a, n, nvars):
    out = {(0,) * nvars: Fraction(1)}
    for _ in range(n):
        out = _pmul(out, a)
    return out


def jacobi_coefficients(n: int, alpha: int) -> list[Fraction]:
    """Coefficients c_i of P_n^{(alpha,0)}(x) = sum_i c_i x^i, from the explicit sum
    P_n^{(a,b)}(x) = sum_s C(n+a, n-s) C(n+b, s) ((x-1)/2)^s ((x+1)/2)^(n-s)."""
    coeffs = [Fraction(0)] * (n + 1)
    xm = {(1,): Fraction(1, 2), (0,): Fraction(-1, 2)}   # (x-1)/2
    xp = {(1,): Fraction(1, 2), (0,): Fraction(1, 2)}    # (x+1)/2
    total = {}
    for s in range(n + 1):
        term = _pmul(_ppow(xm, s, 1), _ppow(xp, n - s, 1))
        total = _padd(total, _pscale(term, comb(n + alpha, n - s) * comb(n, s)))
    for (i,), v in total.items():
        coeffs[i] = Fraction(v)
    return coeffs


def _collapsed_factor(coeffs, u, s, nvars):
    """sum_i c_i (2u - s)^i s^(deg - i): the polynomial P(2u/s - 1) s^deg."""
    deg = len(coeffs) - 1
    two_u_minus_s = _padd(_pscale(u, 2), _pscale(s, -1))
    out = {}
    for i, c in enumerate(coeffs):
        if c == 0:
            continue
        term = _pmul(_ppow(two_u_minus_s, i, nvars), _ppow(s, deg - i, nvars))
        out = _padd(out, _pscale(term, c))
    return out


def tet_indices(order_n: int):
    """(p, q, r) of the tetrahedral basis in library order: degree, then (p, q)."""
    out = []
    for d in range(order_n + 1):
        for p in range(d + 1):
            for q in range(d - p + 1):
                out.append((p, q, d - p - q))
    return out


def tri_indices(order_n: int):
    out = []
    for d in range(order_n + 1):
        for p in range(d + 1):
            out.append((p, d - p))
    return out


@lru_cache(maxsize=None)
def tet_basis_polys(order_n: int):
    """Exact Dubiner polynomials on the reference tetrahedron (list of dicts)."""
    xi = {(1, 0, 0): Fraction(1)}
    eta = {(0, 1, 0): Fraction(1)}
    zeta = {(0, 0, 1): Fraction(1)}
    one = {(0, 0, 0): Fraction(1)}
    s1 = _padd(one, _pscale(_padd(eta, zeta), -1))
    s2 = _padd(one, _pscale(zeta, -1))
    polys = []
    for p, q, r in tet_indices(order_n):
        f1 = _collapsed_factor(jacobi_coefficients(p, 0), xi, s1, 3)
        f2 = _collapsed_factor(jacobi_coefficients(q, 2 * p + 1), eta, s2, 3)
        c3 = jacobi_coefficients(r, 2 * p + 2 * q + 2)
        f3 = {}
        two_z_minus_1 = _padd(_pscale(zeta, 2), _pscale(one, -1))
        for i, c in enumerate(c3):
            f3 = _padd(f3, _pscale(_ppow(two_z_minus_1, i, 3), c))
        polys.append(_pmul(_pmul(f1, f2), f3))
    return polys


@lru_cache(maxsize=None)
def tri_basis_polys(order_n: int):
    c1 = {(1, 0): Fraction(1)}
    c2 = {(0, 1): Fraction(1)}
    one = {(0, 0): Fraction(1)}
    s = _padd(one, _pscale(c2, -1))
    polys = []
    for p, q in tri_indices(order_n):
        f1 = _collapsed_factor(jacobi_coefficients(p, 0), c1, s, 2)
        cq = jacobi_coefficients(q, 2 * p + 1)
        two_c2_minus_1 = _padd(_pscale(c2, 2), _pscale(one, -1))
        f2 = {}
        for i, c in enumerate(cq):
            f2 = _padd(f2, _pscale(_ppow(two_c2_minus_1, i, 2), c))
        polys.append(_pmul(f1, f2))
    return polys


def _monomials3(deg):
    return [(a, b, d - a - b) for d in range(deg + 1) for a in range(d, -1, -1) for b in range(d - a, -1, -1)]


def _monomials2(deg):
    return [(a, d - a) for d in range(deg + 1) for a in range(d, -1, -1)]


def _int_columns(polys, monos):
    """Integer coefficient matrix C (n_mono x n_poly) and per-column denominators."""
    index = {m: i for i, m in enumerate(monos)}
    n = len(polys)
    C = np.zeros((len(monos), n), dtype=object)
    dens = []
    for k, poly in enumerate(polys):
        den = 1
        for v in poly.values():
            den = lcm(den, Fraction(v).denominator)
        dens.append(den)
        for m, v in poly.items():
            C[index[m], k] = int(Fraction(v) * den)
    C[C == 0] = 0
    return C, dens


def _compose_affine(monos3, monos2, maps):
    """T[g, a]: 2D coefficients of the 3D monomial a composed with affine maps.
    maps = three 2D polynomials (dicts) giving xi, eta, zeta as functions of chi."""
    index2 = {m: i for i, m in enumerate(monos2)}
    T = np.zeros((len(monos2), len(monos3)), dtype=object)
    T[:, :] = 0
    for ai, (a, b, c) in enumerate(monos3):
        poly = _pmul(_pmul(_ppow(maps[0], a, 2), _ppow(maps[1], b, 2)), _ppow(maps[2], c, 2))
        for m, v in poly.items():
            assert Fraction(v).denominator == 1
            T[index2[m], ai] = int(v)
    return T


def _face_map(sigma: int, h: int | None = None):
    """Affine map chi -> (xi, eta, zeta) of face sigma (0-based), optionally composed
    with the neighbour orientation Theta_h (the argument of the map is then Theta_h(chi))."""
    c1 = {(1, 0): Fraction(1)}
    c2 = {(0, 1): Fraction(1)}
    one = {(0, 0): Fraction(1)}
    rest = _padd(one, _pscale(_padd(c1, c2), -1))
    if h is None:
        u, v = c1, c2
    elif h == 0:
        u, v = c2, c1
    elif h == 1:
        u, v = rest, c2
    elif h == 2:
        u, v = c1, rest
    else:
        raise ValueError(h)
    va, vb, vc = (TET_VERTICES[i] for i in FACE_VERTICES[sigma])
    comps = []
    for x in range(3):
        poly = {}
        if va[x]:
            poly = _padd(poly, _pscale(one, va[x]))
        if vb[x] - va[x]:
            poly = _padd(poly, _pscale(u, vb[x] - va[x]))
        if vc[x] - va[x]:
            poly = _padd(poly, _pscale(v, vc[x] - va[x]))
        comps.append(poly)
    return comps


def _gram3(monos, L):
    n = len(monos)
    G = np.zeros((n, n), dtype=object)
    for i, (a, b, c) in enumerate(monos):
        for j, (a2, b2, c2) in enumerate(monos):
            A, Bb, Cc = a + a2, b + b2, c + c2
            G[i, j] = L * factorial(A) * factorial(Bb) * factorial(Cc) // factorial(A + Bb + Cc + 3)
    return G


def _gram2(monos, L):
    n = len(monos)
    G = np.zeros((n, n), dtype=object)
    for i, (a, b) in enumerate(monos):
        for j, (a2, b2) in enumerate(monos):
            G[i, j] = L * factorial(a + a2) * factorial(b + b2) // factorial(a + a2 + b + b2 + 2)
    return G


def _to_fraction_matrix(num, row_den, col_den, L):
    r, c = num.shape
    out = np.empty((r, c), dtype=object)
    for i in range(r):
        for j in range(c):
            out[i, j] = Fraction(int(num[i, j]), row_den[i] * col_den[j] * L)
    return out


def to_float(mat) -> np.ndarray:
    """Correctly rounded float64 copy of an exact Fraction array."""
    return np.vectorize(float, otypes=[np.float64])(mat)


@lru_cache(maxsize=None)
def exact_matrices(order_n: int) -> dict:
    """All global matrices of degree-N tetrahedral ADER-DG as exact Fraction arrays.

    Keys: M (B x B), K (3, B, B), Khat, Ktilde (3, B, B), Fm (4, B, B),
    Fp (4, 4, 3, B, B) indexed [sigma, j, h], R (4, B, Bt), W (Bt,), f (3, Bt, Bt),
    Rhat (4, B, Bt), FmHat (4,B,B) = M^-1 Fm, FpHat (4,4,3,B,B) = M^-1 Fp.
    """
    N = order_n
    B, Bt = n_basis(N), n_face_basis(N)
    monos3, monos2 = _monomials3(N), _monomials2(N)
    C, dens = _int_columns(tet_basis_polys(N), monos3)
    Cpsi, dens_psi = _int_columns(tri_basis_polys(N), monos2)
    L3 = factorial(2 * N + 3)
    L2 = factorial(2 * N + 2)
    G3 = _gram3(monos3, L3)
    G2 = _gram2(monos2, L2)

    M = _to_fraction_matrix(C.T.dot(G3).dot(C), dens, dens, L3)
    idx3 = {m: i for i, m in enumerate(monos3)}
    K = np.empty((3, B, B), dtype=object)
    for d in range(3):
        DC = np.zeros_like(C)
        DC[:, :] = 0
        for i, m in enumerate(monos3):
            up = list(m)
            up[d] += 1
            up = tuple(up)
            if up in idx3:
                DC[i, :] = C[idx3[up], :] * up[d]
        K[d] = _to_fraction_matrix(DC.T.dot(G3).dot(C), dens, dens, L3)

    Minv = np.array([1 / M[k, k] for k in range(B)], dtype=object)
    Khat = np.empty_like(K)
    Ktilde = np.empty_like(K)
    for d in range(3):
        Khat[d] = Minv[:, None] * K[d]
        Ktilde[d] = -Minv[:, None] * K[d].T

    U = [_compose_affine(monos3, monos2, _face_map(s)).dot(C) for s in range(4)]
    Uh = [[_compose_affine(monos3, monos2, _face_map(j, h)).dot(C) for h in range(3)] for j in range(4)]
    Fm = np.empty((4, B, B), dtype=object)
    Fp = np.empty((4, 4, 3, B, B), dtype=object)
    for s in range(4):
        GU = G2.dot(U[s])
        Fm[s] = _to_fraction_matrix(U[s].T.dot(GU), dens, dens, L2)
        for j in range(4):
            for h in range(3):
                Fp[s, j, h] = _to_fraction_matrix(U[s].T.dot(G2).dot(Uh[j][h]), dens, dens, L2)

    Wnum = Cpsi.T.dot(G2).dot(Cpsi)
    W = np.array([Fraction(int(Wnum[m, m]), dens_psi[m] ** 2 * L2) for m in range(Bt)], dtype=object)
    R = np.empty((4, B, Bt), dtype=object)
    for s in range(4):
        proj = _to_fraction_matrix(U[s].T.dot(G2).dot(Cpsi), dens, dens_psi, L2)
        R[s] = proj / W[None, :]
    f = np.empty((3, Bt, Bt), dtype=object)
    for h in range(3):
        Tpsi = _compose_psi(monos2, h).dot(Cpsi)   # psi_n o Theta_h, column n
        P = _to_fraction_matrix(Tpsi.T.dot(G2).dot(Cpsi), dens_psi, dens_psi, L2) / W[None, :]
        f[h] = P.T                                  # f_mn = P_nm
    Rhat = np.empty_like(R)
    for s in range(4):
        Rhat[s] = Minv[:, None] * R[s] * W[None, :]
    FmHat = Minv[None, :, None] * Fm
    FpHat = Minv[None, None, None, :, None] * Fp
    return dict(M=M, K=K, Khat=Khat, Ktilde=Ktilde, Fm=Fm, Fp=Fp, R=R, W=W, f=f,
                Rhat=Rhat, FmHat=FmHat, FpHat=FpHat)


def _compose_psi(monos2, h):
    """T[g, a]: 2D monomial a composed with Theta_h, in 2D monomial coefficients."""
    c1 = {(1, 0): Fraction(1)}
    c2 = {(0, 1): Fraction(1)}
    one = {(0, 0): Fraction(1)}
    rest = _padd(one, _pscale(_padd(c1, c2), -1))
    u, v = [(c2, c1), (rest, c2), (c1, rest)][h]
    index2 = {m: i for i, m in enumerate(monos2)}
    T = np.zeros((len(monos2), len(monos2)), dtype=object)
    T[:, :] = 0
    for ai, (a, b) in enumerate(monos2):
        poly = _pmul(_ppow(u, a, 2), _ppow(v, b, 2))
        for m, val in poly.items():
            T[index2[m], ai] = int(val)
    return T


@lru_cache(maxsize=None)
def float_matrices(order_n: int) -> dict:
    """float64 (correctly rounded) copies of ``exact_matrices``."""
    ex = exact_matrices(order_n)
    return {k: to_float(v) for k, v in ex.items()}


def evaluate_tet_basis(order_n: int, points: np.ndarray) -> np.ndarray:
    """phi_k at points (n, 3) -> (n, B), from the exact monomial expansion evaluated in
    float64 with Horner-free direct powers (used only for smooth projections)."""
    polys = tet_basis_polys(order_n)
    pts = np.asarray(points, dtype=np.float64)
    out = np.zeros((pts.shape[0], len(polys)))
    for k, poly in enumerate(polys):
        for (a, b, c), v in poly.items():
            out[:, k] += float(v) * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c
    return out
