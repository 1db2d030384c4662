"""Seeded synthetic inputs shaped like the paper's SeisSol workloads.

This module holds only input generation (random numbers, mesh connectivity, a CFL time
step); none of the scheme's arithmetic.  Both the oracle-based tests and the GPU path's
tests / benchmark draw their inputs from here.

Recipe (stand-in for the SeisSol performance reproducer, which runs on random data with
random neighbour relations, Sec. 6.3, and for the 1.1 M-tet LOH.1 scale, Sec. 6.4):
  * material per element: rho ~ U[2000, 3000], lambda, mu ~ U[1e10, 4e10];
  * affine element map x = x0 + J xi with J = I + 0.3 N(0,1)_{3x3}, redrawn while
    det J <= 0.1;
  * DOFs Q ~ N(0,1) ("unit"), or with the six stress rows scaled by rho c_p so that the
    stress and velocity updates of one step have comparable size ("impedance");
  * connectivity: a random perfect matching of the 4E face slots without self pairs; the
    matched slot gives Neigh and Face (j), the orientation h ~ U{0,1,2};
  * time step dt = 0.5 min_e (h_e / c_p,e) / (2N + 1), h_e the insphere diameter.
All draws come from one numpy PCG64 stream seeded with ``seed`` (default 1903).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED = 1903
FACE_VERTICES = ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3))


@dataclass
class Elements:
    rho: np.ndarray       # (E,)
    lam: np.ndarray       # (E,)
    mu: np.ndarray        # (E,)
    jac: np.ndarray       # (E, 3, 3)   dx/dxi (columns = edge vectors)


@dataclass
class Connectivity:
    neighbours: np.ndarray   # (E, 4) int32
    faces: np.ndarray        # (E, 4) int8   neighbour's face j
    orient: np.ndarray       # (E, 4) int8   orientation h


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_elements(n_elements: int, seed: int = SEED) -> Elements:
    rng = _rng(seed)
    rho = rng.uniform(2000.0, 3000.0, n_elements)
    lam = rng.uniform(1e10, 4e10, n_elements)
    mu = rng.uniform(1e10, 4e10, n_elements)
    jac = np.eye(3)[None] + 0.3 * rng.standard_normal((n_elements, 3, 3))
    bad = np.linalg.det(jac) <= 0.1
    while bad.any():
        jac[bad] = np.eye(3)[None] + 0.3 * rng.standard_normal((int(bad.sum()), 3, 3))
        bad = np.linalg.det(jac) <= 0.1
    return Elements(rho, lam, mu, jac)


def random_dofs(n_elements: int, n_basis: int, seed: int = SEED + 1, scale: str = "unit",
                elements: Elements | None = None) -> np.ndarray:
    """Q (E, B, 9) indexed [element, basis function, quantity]."""
    rng = _rng(seed)
    Q = rng.standard_normal((n_elements, n_basis, 9))
    if scale == "impedance":
        assert elements is not None
        z = elements.rho * np.sqrt((elements.lam + 2 * elements.mu) / elements.rho)
        Q[:, :, :6] *= z[:, None, None]
    elif scale != "unit":
        raise ValueError(scale)
    return Q


def random_connectivity(n_elements: int, seed: int = SEED + 2) -> Connectivity:
    """Random perfect matching of the 4E face slots (no element paired with itself)."""
    if n_elements < 2:
        raise ValueError("need at least two elements")
    rng = _rng(seed)
    slots = rng.permutation(4 * n_elements).astype(np.int64)
    a, b = slots[0::2].copy(), slots[1::2].copy()
    for _ in range(1000):
        self_pair = np.nonzero(a // 4 == b // 4)[0]
        if self_pair.size == 0:
            break
        other = rng.integers(0, a.size, self_pair.size)
        b[self_pair], b[other] = b[other].copy(), b[self_pair].copy()
    else:
        raise RuntimeError("could not remove self pairs")
    nb = np.empty(4 * n_elements, dtype=np.int64)
    nb[a] = b
    nb[b] = a
    neighbours = (nb // 4).reshape(n_elements, 4).astype(np.int32)
    faces = (nb % 4).reshape(n_elements, 4).astype(np.int8)
    orient = rng.integers(0, 3, (n_elements, 4)).astype(np.int8)
    return Connectivity(neighbours, faces, orient)


def insphere_diameter(jac: np.ndarray) -> np.ndarray:
    ref = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    X = np.einsum('eij,vj->evi', jac, ref)
    area = np.zeros(jac.shape[0])
    for fv in FACE_VERTICES:
        a, b, c = X[:, fv[0]], X[:, fv[1]], X[:, fv[2]]
        area += 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=-1)
    volume = np.abs(np.linalg.det(jac)) / 6.0
    return 6.0 * volume / area


def cfl_time_step(elements: Elements, order_n: int, cfl: float = 0.5) -> float:
    cp = np.sqrt((elements.lam + 2 * elements.mu) / elements.rho)
    h = insphere_diameter(elements.jac)
    return float(cfl * np.min(h / cp) / (2 * order_n + 1))


# ----------------------------------------------------------------------- periodic mesh
@dataclass
class Mesh:
    vertices: np.ndarray      # (E, 4, 3) unwrapped physical vertex coordinates
    elements: Elements
    conn: Connectivity
    h: float


def periodic_cube_mesh(n: int, length: float = 1.0, rho=1.0, lam=2.0, mu=1.0) -> Mesh:
    """n^3 cubes of a periodic box, each split into 6 tetrahedra along its main diagonal
    (Kuhn triangulation); homogeneous material; neighbour face j and orientation h found
    by matching shared vertices."""
    if n < 3:
        raise ValueError("n >= 3 keeps the periodic vertex ids of a face distinct")
    h = length / n
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    verts, ids = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                c = np.array([i, j, k])
                for pm in perms:
                    p0 = c.copy()
                    p1 = p0.copy(); p1[pm[0]] += 1
                    p2 = p1.copy(); p2[pm[1]] += 1
                    p3 = c + 1
                    pts = [p0, p1, p2, p3]
                    J = np.stack([pts[1] - pts[0], pts[2] - pts[0], pts[3] - pts[0]], axis=1)
                    if np.linalg.det(J) < 0:
                        pts[1], pts[2] = pts[2], pts[1]
                    verts.append(np.array(pts, dtype=np.float64) * h)
                    ids.append([tuple(int(x) % n for x in p) for p in pts])
    verts = np.array(verts)
    E = verts.shape[0]
    jac = np.stack([verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0],
                    verts[:, 3] - verts[:, 0]], axis=2)
    face_key = {}
    for e in range(E):
        for s, fv in enumerate(FACE_VERTICES):
            key = frozenset(ids[e][v] for v in fv)
            face_key.setdefault(key, []).append((e, s))
    neighbours = np.zeros((E, 4), dtype=np.int32)
    faces = np.zeros((E, 4), dtype=np.int8)
    orient = np.zeros((E, 4), dtype=np.int8)
    for key, lst in face_key.items():
        assert len(lst) == 2, "non-conforming periodic mesh"
        for (e, s), (f, t) in (lst, lst[::-1]):
            local = [ids[e][v] for v in FACE_VERTICES[s]]
            other = [ids[f][v] for v in FACE_VERTICES[t]]
            hh = local.index(other[0])
            expect = [[local[0], local[2], local[1]], [local[1], local[0], local[2]],
                      [local[2], local[1], local[0]]][hh]
            assert other == expect, "inconsistent face orientation"
            neighbours[e, s], faces[e, s], orient[e, s] = f, t, hh
    el = Elements(np.full(E, float(rho)), np.full(E, float(lam)), np.full(E, float(mu)), jac)
    return Mesh(verts, el, Connectivity(neighbours, faces, orient), h)
