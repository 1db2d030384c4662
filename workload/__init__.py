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


@dataclass
class Attenuation:
    omega: np.ndarray     # (E, 3) relaxation frequencies of the three mechanisms
    ylam: np.ndarray      # (E, 3) anelastic moduli Y^lambda_l
    ymu: np.ndarray       # (E, 3) anelastic moduli Y^mu_l


def attenuation(elements: Elements, dt: float, seed: int = SEED + 900,
                omega_dt=(0.005, 0.05, 0.5), y: float = 0.02) -> Attenuation:
    """Synthetic parameters of three attenuation mechanisms per element (the paper gives
    none): omega_l dt = omega_dt[l] x U[0.8, 1.25] (a band of two decades around
    omega dt = 0.05, so that relaxation is resolved by the step), Y_l = y x U[0.5, 1.5] x
    (lambda, mu) (a weak attenuation, quality factor of order 1 / y)."""
    rng = _rng(seed)
    E = elements.rho.shape[0]
    omega = np.asarray(omega_dt)[None, :] * rng.uniform(0.8, 1.25, (E, 3)) / dt
    fy = y * rng.uniform(0.5, 1.5, (E, 3))
    return Attenuation(omega, fy * elements.lam[:, None], fy * elements.mu[:, None])


def random_dofs_viscoelastic(n_elements: int, n_basis: int, elements: Elements,
                             att: Attenuation, seed: int = SEED + 901) -> np.ndarray:
    """Q (E, B, 27): elastic part as random_dofs(..., "impedance"); the anelastic
    functions of mechanism l (units of stress per time) ~ N(0,1) rho c_p omega_l, so that
    their feedback into the stresses over one step is of the size of the elastic
    increment."""
    rng = _rng(seed)
    Q = rng.standard_normal((n_elements, n_basis, 27))
    z = elements.rho * np.sqrt((elements.lam + 2 * elements.mu) / elements.rho)
    Q[:, :, :6] *= z[:, None, None]
    for l in range(3):
        Q[:, :, 9 + 6 * l:15 + 6 * l] *= (z * att.omega[:, l])[:, None, None]
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
        # one swap at a time: a permutation also when the draws repeat or hit a self pair
        for i, o in zip(self_pair, other):
            b[i], b[o] = b[o], b[i]
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


_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
_ROTATIONS = np.array([[0, 2, 1], [1, 0, 2], [2, 1, 0]])


def jittered_periodic_mesh(n: int, jitter: float = 0.0, seed: int = SEED + 800,
                           length: float = 1.0, rho=1.0, lam=2.0, mu=1.0) -> Mesh:
    """The mesh of ``periodic_cube_mesh`` built with array operations (n = 55 gives
    998,250 tets in seconds), with every periodic vertex moved by jitter * h * U[-1, 1]^3
    (one displacement per periodic vertex id, so that the periodic images of a vertex
    move together and the mesh stays conforming).  jitter = 0 reproduces
    ``periodic_cube_mesh`` element by element."""
    if n < 3:
        raise ValueError("n >= 3 keeps the periodic vertex ids of a face distinct")
    h = length / n
    g = np.arange(n)
    corner = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 1, 3)
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for pm in _KUHN_PERMS:
        p1 = unit[pm[0]]
        p2 = p1 + unit[pm[1]]
        order = [0, 1, 2, 3]
        if np.linalg.det(np.stack([p1, p2, np.ones(3)], axis=1)) < 0:
            order = [0, 2, 1, 3]
        local = np.stack([np.zeros(3, np.int64), p1, p2, np.ones(3, np.int64)])[order]
        tets.append(local)
    lattice = corner[:, None] + np.stack(tets)[None]            # (n^3, 6, 4, 3)
    lattice = lattice.reshape(-1, 4, 3)
    E = lattice.shape[0]
    wrapped = lattice % n
    ids = (wrapped[..., 0] * n + wrapped[..., 1]) * n + wrapped[..., 2]    # (E, 4)
    verts = lattice.astype(np.float64) * h
    if jitter > 0.0:
        disp = _rng(seed).uniform(-1.0, 1.0, (n ** 3, 3)) * (jitter * h)
        verts = verts + disp[ids]
    jac = np.stack([verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0],
                    verts[:, 3] - verts[:, 0]], axis=2)
    if not (np.linalg.det(jac) > 0).all():
        raise ValueError("jitter too large: an element is inverted")
    fv = np.array(FACE_VERTICES)
    face_ids = ids[:, fv]                                       # (E, 4, 3)
    s = np.sort(face_ids, axis=-1).reshape(-1, 3).astype(np.int64)
    key = (s[:, 0] * n ** 3 + s[:, 1]) * n ** 3 + s[:, 2]
    perm = np.argsort(key, kind="stable")
    a, b = perm[0::2], perm[1::2]
    if not (key[a] == key[b]).all() or (a.size > 1 and (key[a[1:]] == key[b[:-1]]).any()):
        raise AssertionError("non-conforming periodic mesh")
    slot = face_ids.reshape(-1, 3)
    neighbours = np.empty(4 * E, np.int32)
    faces = np.empty(4 * E, np.int8)
    orient = np.empty(4 * E, np.int8)
    for x, y in ((a, b), (b, a)):
        loc, oth = slot[x], slot[y]
        hh = np.argmax(loc == oth[:, :1], axis=1)
        expect = np.take_along_axis(loc, _ROTATIONS[hh], axis=1)
        if not (expect == oth).all():
            raise AssertionError("inconsistent face orientation")
        neighbours[x] = y // 4
        faces[x] = y % 4
        orient[x] = hh
    el = Elements(np.full(E, float(rho)), np.full(E, float(lam)), np.full(E, float(mu)), jac)
    conn = Connectivity(neighbours.reshape(E, 4), faces.reshape(E, 4), orient.reshape(E, 4))
    return Mesh(verts, el, conn, h)
