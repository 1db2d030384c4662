"""Tensor-core form (YT_BF16X3_F32ACC) of the step against the FP64 oracle.

Products with the global matrices use split bf16 operands (hi + lo, three products,
binary32 accumulation): each such product carries a relative error of about 2^-16 of
|a||x|, so the bounds below are stated per quantity in the relative Frobenius norm, for
the time integral and for the increment Q_new - Q (the part of Q a step changes)."""
import numpy as np
import pytest

import parity
import workload as wl
from oracle import basis, planewave, scheme

pytestmark = pytest.mark.gpu

TC_TOL_I = parity.TC_I            # time integral
TC_TOL_INCREMENT = parity.TC_INC  # Q_new - Q


@pytest.fixture(scope="module")
def yt():
    import paper_1903_11521_gb300 as yt
    yt.load()
    return yt


def rel_per_quantity(a, b):
    num = np.sqrt(((a - b) ** 2).sum(axis=(0, 1)))
    den = np.sqrt((b ** 2).sum(axis=(0, 1)))
    return num / den


def make_case(E, order, scale, seed):
    N = order - 1
    el = wl.random_elements(E, seed=seed)
    conn = wl.random_connectivity(E, seed=seed + 2)
    Q = wl.random_dofs(E, basis.n_basis(N), seed=seed + 1, scale=scale, elements=el)
    dt = wl.cfl_time_step(el, N)
    return el, conn, Q, dt


def solver(yt, el, conn, Q, dt, order):
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient,
                  precision=yt.YT_BF16X3_F32ACC)
    s.set_dofs_host(Q)
    return s


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_tc_full_step_against_fp64_oracle(yt, order):
    el, conn, Q, dt = make_case(70, order, "impedance", seed=41)
    s = solver(yt, el, conn, Q, dt, order)
    s.step()
    s.status()
    q, i = s.get_host(yt.YT_FIELD_DOFS), s.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    s.close()
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    q_ref, I = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient,
                                dt, order - 1)
    parity.check(f"tc step o{order} I", i, I, TC_TOL_I, parity.TC_I_EL)
    parity.check(f"tc step o{order} dQ", q, q_ref, TC_TOL_INCREMENT, parity.TC_INC_EL, base=Q)


@pytest.mark.parametrize("order", [3, 6, 7])
def test_tc_local_step(yt, order):
    """yt_step_local: k_local_tc, then the lifting kernel with the local products only."""
    el, conn, Q, dt = make_case(45, order, "unit", seed=43)
    s = solver(yt, el, conn, Q, dt, order)
    s.step_local()
    s.status()
    q, i = s.get_host(yt.YT_FIELD_DOFS), s.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    s.close()
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    _, I = scheme.derivatives_and_time_integral(Q, star, dt, order - 1)
    q_ref = scheme.local_update(Q, I, star, loc, order - 1)
    parity.check(f"tc local o{order} I", i, I, TC_TOL_I, parity.TC_I_EL)
    parity.check(f"tc local o{order} dQ", q, q_ref, TC_TOL_INCREMENT, parity.TC_INC_EL, base=Q)


@pytest.mark.parametrize("order", [4, 7])
def test_tc_many_tiles_and_phases(yt, order):
    """More tiles than persistent CTAs (each CTA strides over several tiles: at order 7
    every tile reloads the streamed operands), a ragged last tile; yt_step equals phase 0
    + phase 1 bitwise, and local + neighbour agrees."""
    el, conn, Q, dt = make_case(152 * 32 * 2 + 17, order, "impedance", seed=47)
    outs = []
    for mode in ("step", "phases", "unfused"):
        s = solver(yt, el, conn, Q, dt, order)
        if mode == "step":
            s.step()
        elif mode == "phases":
            s.step_phase(0)
            s.step_phase(1)
        else:
            s.step_local()
            s.step_neighbour()
        s.status()
        outs.append(s.get_host())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    q_ref, _ = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient,
                                dt, order - 1)
    for mode, out in zip(("step", "phases", "unfused"), outs):
        parity.check(f"tc many tiles {mode} dQ", out, q_ref, TC_TOL_INCREMENT, parity.TC_INC_EL, base=Q)


def test_tc_deterministic(yt):
    el, conn, Q, dt = make_case(64, 5, "unit", seed=49)
    res = []
    for _ in range(2):
        s = solver(yt, el, conn, Q, dt, 5)
        s.step()
        res.append(s.get_host())
        s.close()
    assert np.array_equal(res[0], res[1])


def test_tc_plane_wave_100_steps(yt):
    """100 steps at order 5 on the periodic mesh: drift from the FP64 path within a stated
    bound (1e-2 per quantity, measured 3.8e-3: the quantities of zero exact amplitude carry
    the largest relative drift; 3e-4 per element, measured 3.5e-5), plane-wave error equal
    to the FP64 one to 5e-2 relative."""
    order, N = 5, 4
    k = 2 * np.pi * np.array([1.0, 1.0, 0.0])
    mesh = wl.periodic_cube_mesh(3)
    el = mesh.elements
    dt = wl.cfl_time_step(el, N, cfl=0.3)
    T = 100 * dt
    Q0 = planewave.project(mesh, N, 0.0, k, 1.0, 2.0, 1.0)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    out = {}
    for prec in (yt.YT_F64, yt.YT_BF16X3_F32ACC):
        s = yt.Solver(order, dt, mat, el.jac, mesh.conn.neighbours, mesh.conn.faces,
                      mesh.conn.orient, precision=prec)
        s.set_dofs_host(Q0)
        for _ in range(100):
            s.step()
        s.status()
        out[prec] = s.get_host()
        s.close()
    drift = rel_per_quantity(out[yt.YT_BF16X3_F32ACC], out[yt.YT_F64]).max()
    el_drift = parity.per_element(out[yt.YT_BF16X3_F32ACC], out[yt.YT_F64]).max()
    print(f"PARITY tc plane wave 100 steps drift {drift:.3e} (bound 1e-2), per-element {el_drift:.3e} (bound 3e-4)")
    assert drift < 1e-2
    assert el_drift < 3e-4
    e64 = planewave.l2_error(mesh, N, out[yt.YT_F64], T, k, 1.0, 2.0, 1.0)
    etc = planewave.l2_error(mesh, N, out[yt.YT_BF16X3_F32ACC], T, k, 1.0, 2.0, 1.0)
    print("plane-wave error fp64", e64, "tensor-core", etc)
    assert np.allclose(etc, e64, rtol=5e-2)


def test_bounded_wait_runs_out_and_reports_timeout(yt):
    """The timeout path of the bounded device waits, without a fault or a hang: with the
    diagnostics flag the tensor-core local kernel issues no operand load, so its first
    wait (limit 1 ms) runs out with nothing in flight; the kernel stops, frees its tensor
    memory and records the timeout.  yt_solver_status reports YT_ERR_TIMEOUT once (and
    clears it); the context stays usable: a fresh solver then steps correctly."""
    order = 4
    el, conn, Q, dt = make_case(70, order, "impedance", seed=45)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient,
                  precision=yt.YT_BF16X3_F32ACC, flags=yt.YT_SCHEME_DIAG_EXPIRE_WAIT)
    s.set_dofs_host(Q)
    s.step()
    with pytest.raises(yt.YtError) as info:
        s.status()
    assert info.value.status == 7
    s.status()                   # the record was cleared
    s.close()
    with pytest.raises(yt.YtError) as info:   # the flag belongs to the tensor-core form
        yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient,
                  precision=yt.YT_F64, flags=yt.YT_SCHEME_DIAG_EXPIRE_WAIT)
    assert info.value.status == 1
    s = solver(yt, el, conn, Q, dt, order)
    s.step()
    s.status()
    q = s.get_host()
    s.close()
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    q_ref, _ = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient,
                                dt, order - 1)
    parity.check("tc after timeout dQ", q, q_ref, TC_TOL_INCREMENT, parity.TC_INC_EL, base=Q)
