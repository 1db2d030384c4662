"""Serving form: continuous batching of independent solves.  Each result must equal the
same solve run alone (bitwise: every tile is computed exactly as alone), admission must
respect the HBM budget, and requests must actually share the device."""
import numpy as np
import pytest

import parity
import workload as wl
from oracle import basis, scheme

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def yt():
    import paper_1903_11521_gb300 as yt
    yt.load()
    return yt


def make_request(seed, order, E):
    el = wl.random_elements(E, seed=seed)
    conn = wl.random_connectivity(E, seed=seed + 1)
    Q = wl.random_dofs(E, basis.n_basis(order - 1), seed=seed + 2, scale="impedance", elements=el)
    dt = wl.cfl_time_step(el, order - 1)
    mat = np.stack([el.rho, el.lam, el.mu], 1)
    return dict(order=order, dt=dt, material=mat, jacobian=el.jac, neighbours=conn.neighbours,
                faces=conn.faces, orient=conn.orient, Q=Q)


def solo(yt, r, steps, precision):
    s = yt.Solver(r['order'], r['dt'], r['material'], r['jacobian'], r['neighbours'],
                  r['faces'], r['orient'], precision=precision)
    s.set_dofs_host(r['Q'])
    for _ in range(steps):
        s.step()
    out = s.get_host()
    s.close()
    return out


def test_mix_equals_alone_and_budget_respected(yt):
    rng = np.random.default_rng(90)
    reqs = []
    for i in range(10):
        order = int(rng.integers(3, 7))
        E = int(rng.integers(2000, 8000))
        steps = int(rng.integers(40, 80))     # long enough that solves overlap in time
        reqs.append((make_request(1000 + 10 * i, order, E), steps))
    budget = 400 * 2 ** 20          # about half of the ten requests at once
    srv = yt.Server(budget, precision=yt.YT_F32)
    ids = [srv.submit(r['order'], r['dt'], r['material'], r['jacobian'], r['neighbours'],
                      r['faces'], r['orient'], r['Q'], steps) for r, steps in reqs]
    results = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st['completed'] == len(reqs) and st['failed'] == 0
    assert 0 < st['peak_bytes'] <= budget
    assert st['max_active'] >= 2
    for (r, steps), (q, lat, queue) in zip(reqs, results):
        assert lat > 0 and 0 <= queue <= lat
        assert np.array_equal(q, solo(yt, r, steps, yt.YT_F32))


def test_fp64_server_matches_oracle(yt):
    r = make_request(2000, 4, 300)
    srv = yt.Server(2 ** 30, precision=yt.YT_F64)
    rid = srv.submit(r['order'], r['dt'], r['material'], r['jacobian'], r['neighbours'], r['faces'],
                     r['orient'], r['Q'], 1)
    q, _, _ = srv.wait(rid)
    srv.close()
    el = wl.Elements(r['material'][:, 0], r['material'][:, 1], r['material'][:, 2], r['jacobian'])
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref, _ = scheme.ader_step(r['Q'], star, loc, nb, r['neighbours'], r['faces'], r['orient'],
                              r['dt'], 3)
    parity.check("server f64 Q", q, ref, parity.F64, parity.F64)
    parity.check("server f64 dQ", q, ref, parity.F64_INC, parity.F64_INC, base=r['Q'])


def test_request_above_budget_fails(yt):
    r = make_request(3000, 5, 2000)
    srv = yt.Server(1 << 20, precision=yt.YT_F32)
    rid = srv.submit(r['order'], r['dt'], r['material'], r['jacobian'], r['neighbours'], r['faces'],
                     r['orient'], r['Q'], 2)
    with pytest.raises(yt.YtError) as info:
        srv.wait(rid)
    assert info.value.status == 5
    srv.close()


def test_failed_step_releases_everything(yt):
    """A step that fails (injected on the host: the worker treats its step 2 as a failed
    CUDA call; nothing faults on the device) ends the server's service: every active
    and pending request fails with YT_ERR_CUDA, its waiter returns, the budget is given
    back, later submissions are refused, and destroy returns."""
    reqs = [make_request(4000 + 10 * i, 3 + i % 3, 300 + 50 * i) for i in range(6)]
    budget = 24 * 2 ** 20          # about four of these (4-12 MB each) at a time; the rest wait
    srv = yt.Server(budget, precision=yt.YT_F32)
    srv.fail_tick(2)
    ids = []
    for r in reqs:
        try:
            ids.append(srv.submit(r['order'], r['dt'], r['material'], r['jacobian'], r['neighbours'],
                                  r['faces'], r['orient'], r['Q'], 50))
        except yt.YtError as e:      # the failure came before this submission: refused
            assert e.status == 6
    assert ids
    for rid in ids:
        with pytest.raises(yt.YtError) as info:
            srv.wait(rid)
        assert info.value.status == 6
    st = srv.stats()
    assert st['failed'] == len(ids) and st['completed'] == 0
    assert st['active'] == 0 and st['pending'] == 0
    r = reqs[0]
    with pytest.raises(yt.YtError) as info:
        srv.submit(r['order'], r['dt'], r['material'], r['jacobian'], r['neighbours'], r['faces'],
                   r['orient'], r['Q'], 1)
    assert info.value.status == 6
    srv.close()
    # a fresh server on the same device still computes the right result
    srv = yt.Server(2 ** 30, precision=yt.YT_F32)
    rid = srv.submit(r['order'], r['dt'], r['material'], r['jacobian'], r['neighbours'], r['faces'],
                     r['orient'], r['Q'], 2)
    q, _, _ = srv.wait(rid)
    srv.close()
    assert np.array_equal(q, solo(yt, r, 2, yt.YT_F32))
