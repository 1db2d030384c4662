"""Input generators: the array-built jittered periodic mesh against the loop-built one and
against the geometry it must have (conforming, periodic, positively oriented)."""
import numpy as np
import pytest

import workload as wl


@pytest.mark.parametrize("n", [3, 4])
def test_unjittered_equals_loop_built_mesh(n):
    a = wl.periodic_cube_mesh(n)
    b = wl.jittered_periodic_mesh(n)
    assert np.array_equal(a.vertices, b.vertices)
    assert np.array_equal(a.elements.jac, b.elements.jac)
    for f in ("neighbours", "faces", "orient"):
        assert np.array_equal(getattr(a.conn, f), getattr(b.conn, f)), f


@pytest.mark.parametrize("n", [3, 5])
def test_jittered_mesh_geometry(n):
    m = wl.jittered_periodic_mesh(n, jitter=0.15, seed=7)
    E = m.vertices.shape[0]
    assert E == 6 * n ** 3
    # volumes positive and summing to the box
    det = np.linalg.det(m.elements.jac)
    assert (det > 0).all()
    assert np.isclose(det.sum() / 6.0, 1.0, rtol=1e-12)
    nb, fj, oh = m.conn.neighbours, m.conn.faces, m.conn.orient
    fv = np.array(wl.FACE_VERTICES)
    rot = np.array([[0, 2, 1], [1, 0, 2], [2, 1, 0]])
    for e in range(E):
        for s in range(4):
            f, t, h = nb[e, s], fj[e, s], oh[e, s]
            assert f != e
            # partner relation is symmetric
            assert nb[f, t] == e and fj[f, t] == s and oh[f, t] == h
            mine = m.vertices[e, fv[s]]
            other = m.vertices[f, fv[t]]
            # the neighbour lists the shared vertices in the rotated reverse order; the
            # coordinates agree up to one periodic translation of the whole face
            shift = other - mine[rot[h]]
            assert np.allclose(shift, shift[0], atol=1e-12)
            assert np.allclose(shift[0], np.round(shift[0]), atol=1e-12)


def test_jitter_is_seeded():
    a = wl.jittered_periodic_mesh(3, jitter=0.1, seed=11)
    b = wl.jittered_periodic_mesh(3, jitter=0.1, seed=11)
    c = wl.jittered_periodic_mesh(3, jitter=0.1, seed=12)
    assert np.array_equal(a.vertices, b.vertices)
    assert not np.array_equal(a.vertices, c.vertices)


@pytest.mark.parametrize("E, seed", [(45, 508), (2, 1), (3, 7), (64, 3), (1000, 1905)])
def test_random_connectivity_is_an_involution(E, seed):
    """Every face slot is paired with exactly one other slot of another element, and the
    pairing is symmetric (the neighbour's neighbour is the element itself)."""
    c = wl.random_connectivity(E, seed=seed)
    assert c.neighbours.min() >= 0 and c.neighbours.max() < E
    assert (c.neighbours != np.arange(E)[:, None]).all()
    assert ((c.faces >= 0) & (c.faces < 4)).all()
    back = c.neighbours[c.neighbours, c.faces]
    assert (back == np.arange(E)[:, None]).all()
    assert (c.faces[c.neighbours, c.faces] == np.arange(4)[None, :]).all()
