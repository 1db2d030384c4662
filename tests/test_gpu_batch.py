"""p-adaptive batches (per-element orders, one CUDA-graph launch per step) against the
oracle's mixed-order step."""
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


def case(E, lo, hi, seed):
    el = wl.random_elements(E, seed=seed)
    conn = wl.random_connectivity(E, seed=seed + 1)
    rng = np.random.default_rng(seed + 2)
    orders = rng.integers(lo, hi + 1, E)
    Q = [wl.random_dofs(1, basis.n_basis(int(o) - 1), seed=seed + 3 + e, scale="impedance",
                        elements=wl.Elements(el.rho[e:e + 1], el.lam[e:e + 1], el.mu[e:e + 1],
                                             el.jac[e:e + 1]))[0] for e, o in enumerate(orders)]
    dt = wl.cfl_time_step(el, int(orders.max()) - 1)
    return el, conn, orders, Q, dt


def rel(a_list, b_list):
    a = np.concatenate([x.ravel() for x in a_list])
    b = np.concatenate([x.ravel() for x in b_list])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def per_quantity(a_list, b_list):
    a = np.concatenate(a_list, axis=0)
    b = np.concatenate(b_list, axis=0)
    return np.sqrt(((a - b) ** 2).sum(0) / (b ** 2).sum(0))


def batch_run(yt, el, conn, orders, Q, dt, precision, steps=1, tune=False):
    b = yt.Batch(orders, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, conn.neighbours,
                 conn.faces, conn.orient, precision=precision)
    b.set_dofs_host(Q)
    chosen = b.tune(3) if tune else None
    for _ in range(steps):
        b.step()
    q = b.get_host()
    i = b.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    st = b.stats()
    b.close()
    return q, i, chosen, st


def test_mixed_orders_fp64(yt):
    el, conn, orders, Q, dt = case(150, 2, 6, 50)
    q, i, _, st = batch_run(yt, el, conn, orders, Q, dt, yt.YT_F64)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref, I = scheme.ader_step_mixed(Q, orders - 1, star, loc, nb, conn.neighbours, conn.faces,
                                    conn.orient, dt)
    assert st['groups'] == 5
    parity.check(f"batch f64 o{orders.min()}-{orders.max()} I", i, I, parity.F64, parity.F64)
    parity.check(f"batch f64 o{orders.min()}-{orders.max()} dQ", q, ref, parity.F64_INC, parity.F64_INC, base=Q)


def test_mixed_orders_fp64_up_to_order7(yt):
    el, conn, orders, Q, dt = case(120, 3, 7, 61)
    q, i, _, st = batch_run(yt, el, conn, orders, Q, dt, yt.YT_F64)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref, I = scheme.ader_step_mixed(Q, orders - 1, star, loc, nb, conn.neighbours, conn.faces,
                                    conn.orient, dt)
    assert st['groups'] == 5
    parity.check(f"batch f64 o{orders.min()}-{orders.max()} I", i, I, parity.F64, parity.F64)
    parity.check(f"batch f64 o{orders.min()}-{orders.max()} dQ", q, ref, parity.F64_INC, parity.F64_INC, base=Q)


def test_mixed_orders_fp32_up_to_order7(yt):
    el, conn, orders, Q, dt = case(120, 3, 7, 60)
    q, i, _, _ = batch_run(yt, el, conn, orders, Q, dt, yt.YT_F32)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref, I = scheme.ader_step_mixed(Q, orders - 1, star, loc, nb, conn.neighbours, conn.faces,
                                    conn.orient, dt)
    parity.check("batch f32 o3-7 I", i, I, parity.F32_I, parity.F32_I_EL)
    parity.check("batch f32 o3-7 dQ", q, ref, parity.F32_INC, parity.F32_INC_EL, base=Q)


def test_uniform_batch_equals_solver(yt):
    el, conn, _, _, dt = case(64, 5, 5, 70)
    Q = wl.random_dofs(64, basis.n_basis(4), seed=71, scale="impedance", elements=el)
    q, _, _, _ = batch_run(yt, el, conn, np.full(64, 5), list(Q), dt, yt.YT_F64, steps=2)
    s = yt.Solver(5, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, conn.neighbours,
                  conn.faces, conn.orient)
    s.set_dofs_host(Q)
    s.step()
    s.step()
    ref = s.get_host()
    s.close()
    assert np.array_equal(np.array(q), ref)


def test_tuner_keeps_state_and_result(yt):
    el, conn, orders, Q, dt = case(200, 3, 6, 80)
    a, _, chosen, _ = batch_run(yt, el, conn, orders, Q, dt, yt.YT_F64, steps=2, tune=True)
    b, _, _, _ = batch_run(yt, el, conn, orders, Q, dt, yt.YT_F64, steps=2)
    assert chosen in (0, 1, 2)
    assert rel(a, b) < 1e-15


def _run_form(yt, el, conn, orders, Q, dt, precision, form, order, chunk, steps):
    b = yt.Batch(orders, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, conn.neighbours,
                 conn.faces, conn.orient, precision=precision)
    b.set_form(form, order, chunk)
    cfg = b.config()
    b.set_dofs_host(Q)
    for _ in range(steps):
        b.step()
    b.status()
    q = b.get_host()
    i = b.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    b.close()
    return q, i, cfg


@pytest.mark.parametrize("order, chunk", [(0, 1), (0, 4), (1, 2)])
def test_persistent_kernel_fp64_equals_kernels_and_oracle(yt, order, chunk):
    """The persistent kernel (one cooperative launch per step: local phase of all groups,
    grid barrier, neighbour phase) computes every tile with the same code as the
    per-degree kernels: bitwise the same result in FP64, for both item orders and
    several claim sizes; and it matches the oracle's mixed-order step."""
    el, conn, orders, Q, dt = case(700, 2, 7, 90)
    ref_q, ref_i, _ = _run_form(yt, el, conn, orders, Q, dt, yt.YT_F64, 0, 0, 1, 1)
    q, i, cfg = _run_form(yt, el, conn, orders, Q, dt, yt.YT_F64, 2, order, chunk, 1)
    print("PARITY persistent batch form:", cfg)
    assert "persistent kernel" in cfg
    for a, c in zip(q, ref_q):
        assert np.array_equal(a, c)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    oq, oI = scheme.ader_step_mixed(Q, orders - 1, star, loc, nb, conn.neighbours, conn.faces,
                                    conn.orient, dt)
    parity.check(f"persistent f64 order{order} chunk{chunk} I", i, oI, parity.F64, parity.F64)
    parity.check(f"persistent f64 order{order} chunk{chunk} dQ", q, oq, parity.F64_INC, parity.F64_INC, base=Q)


def test_persistent_kernel_fp32_and_several_steps(yt):
    """FP32 contractions in the persistent kernel (values of the sparse rows from global
    memory instead of constant memory): equal to the per-degree kernels within the FP32
    bounds after three steps, and within them of the oracle after one step."""
    el, conn, orders, Q, dt = case(500, 3, 7, 95)
    ref3, _, _ = _run_form(yt, el, conn, orders, Q, dt, yt.YT_F32, 0, 0, 1, 3)
    got3, _, _ = _run_form(yt, el, conn, orders, Q, dt, yt.YT_F32, 2, 0, 2, 3)
    exact = all(np.array_equal(a, c) for a, c in zip(got3, ref3))
    print(f"PARITY persistent f32 3 steps bitwise equal to the per-degree kernels: {exact}")
    parity.check("persistent f32 vs kernels 3 steps dQ", got3, ref3, parity.F32_INC, parity.F32_INC_EL, base=Q)
    q1, i1, _ = _run_form(yt, el, conn, orders, Q, dt, yt.YT_F32, 2, 1, 1, 1)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    oq, oI = scheme.ader_step_mixed(Q, orders - 1, star, loc, nb, conn.neighbours, conn.faces,
                                    conn.orient, dt)
    parity.check("persistent f32 I", i1, oI, parity.F32_I, parity.F32_I_EL)
    parity.check("persistent f32 dQ", q1, oq, parity.F32_INC, parity.F32_INC_EL, base=Q)
