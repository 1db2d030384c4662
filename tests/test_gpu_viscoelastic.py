"""27-quantity (viscoelastic-shaped) step on the device against the oracle of
oracle/viscoelastic.py: FP64 within 1e-12 (per quantity and per element, the nine
elastic quantities and the eighteen anelastic functions alike), FP32 and the split-bf16
tensor-core form within the bounds of tests/parity.py; yt_step = phase 0 + phase 1 and =
yt_step_host bitwise; several steps on the jittered structured mesh; degenerate inputs."""
import numpy as np
import pytest

import parity
import workload as wl
from oracle import basis
from oracle import viscoelastic as ve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def yt():
    import paper_1903_11521_gb300 as yt
    yt.load()
    return yt


def make_case(E, order, seed):
    N = order - 1
    el = wl.random_elements(E, seed=seed)
    conn = wl.random_connectivity(E, seed=seed + 1)
    dt = wl.cfl_time_step(el, N)
    att = wl.attenuation(el, dt, seed=seed + 2)
    Q = wl.random_dofs_viscoelastic(E, basis.n_basis(N), el, att, seed=seed + 3)
    return el, conn, dt, att, Q


def solver(yt, el, conn, dt, att, order, precision):
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    return yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient,
                     precision=precision, attenuation=att)


def oracle_steps(el, conn, dt, att, Q, order, steps=1):
    star, src, loc, nb = ve.setup_element_matrices(el.rho, el.lam, el.mu, att.ylam, att.ymu,
                                                   att.omega, el.jac)
    I = None
    for _ in range(steps):
        Q, I = ve.ader_step(Q, star, src, loc, nb, conn.neighbours, conn.faces, conn.orient, dt,
                            order - 1)
    return Q, I


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_ve_fp64_step_against_oracle(yt, order):
    E = 70 if order < 7 else 45
    el, conn, dt, att, Q = make_case(E, order, 500 + order)
    s = solver(yt, el, conn, dt, att, order, yt.YT_F64)
    s.set_dofs_host(Q)
    s.step()
    q, i = s.get_host(), s.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    s.close()
    q_ref, I_ref = oracle_steps(el, conn, dt, att, Q, order)
    parity.check(f"ve f64 o{order} I", i, I_ref, parity.F64, parity.F64)
    parity.check(f"ve f64 o{order} Q", q, q_ref, parity.F64, parity.F64)
    parity.check(f"ve f64 o{order} dQ", q, q_ref, parity.F64_INC, parity.F64_INC, base=Q)


@pytest.mark.parametrize("order", [2, 4, 6, 7])
def test_ve_fp32_step_against_oracle(yt, order):
    el, conn, dt, att, Q = make_case(70, order, 520 + order)
    s = solver(yt, el, conn, dt, att, order, yt.YT_F32)
    s.set_dofs_host(Q)
    s.step()
    q, i = s.get_host(), s.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    s.close()
    q_ref, I_ref = oracle_steps(el, conn, dt, att, Q, order)
    parity.check(f"ve f32 o{order} I", i, I_ref, parity.VE_F32_I, parity.VE_F32_I_EL)
    parity.check(f"ve f32 o{order} dQ", q, q_ref, parity.VE_F32_INC, parity.VE_F32_INC_EL, base=Q)


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_ve_bf16x3_step_against_oracle(yt, order):
    """Tensor-core form: the elastic rows' global-matrix products in split bf16 (every
    derivative on the first derivative's passes, all B rows), the anelastic functions on
    the CUDA cores in FP32, binary64 time integral and updates."""
    E = 70 if order < 7 else 45
    el, conn, dt, att, Q = make_case(E, order, 580 + order)
    s = solver(yt, el, conn, dt, att, order, yt.YT_BF16X3_F32ACC)
    s.set_dofs_host(Q)
    s.step()
    q, i = s.get_host(), s.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    s.status()
    s.close()
    q_ref, I_ref = oracle_steps(el, conn, dt, att, Q, order)
    parity.check(f"ve bf16x3 o{order} I", i, I_ref, parity.VE_TC_I, parity.VE_TC_I_EL)
    parity.check(f"ve bf16x3 o{order} dQ", q, q_ref, parity.VE_TC_INC, parity.VE_TC_INC_EL, base=Q)


@pytest.mark.parametrize("prec_name", ["YT_F64", "YT_F32", "YT_BF16X3_F32ACC"])
def test_ve_phases_and_host_step_equal_step(yt, prec_name):
    """yt_step == phase 0 + phase 1 and == yt_step_host (element chunks, ragged last
    chunk and tile) bitwise."""
    import torch
    prec = getattr(yt, prec_name)
    order = 4
    E = 8 * 32 * 3 + 45
    el, conn, dt, att, Q = make_case(E, order, 540)
    outs = []
    for mode in ("step", "phases"):
        s = solver(yt, el, conn, dt, att, order, prec)
        s.set_dofs_host(Q)
        if mode == "step":
            s.step()
        else:
            s.step_phase(0)
            s.step_phase(1)
        outs.append(s.get_host())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    s = solver(yt, el, conn, dt, att, order, prec)
    canon = np.ascontiguousarray(Q.transpose(0, 2, 1))
    pin_in = torch.from_numpy(canon.copy()).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    s.step_host_ptr(pin_in.data_ptr(), pin_out.data_ptr())
    torch.cuda.synchronize()
    s.close()
    assert np.array_equal(pin_out.numpy().transpose(0, 2, 1), outs[0])


@pytest.mark.parametrize("prec_name, order, tol, tol_el", [
    ("YT_F64", 7, 1e-12, 1e-11), ("YT_F32", 7, None, None), ("YT_BF16X3_F32ACC", 7, "tc", None)])
def test_ve_jittered_mesh_three_steps(yt, prec_name, order, tol, tol_el):
    """Three steps on the jittered periodic structured mesh (the mesh family of the
    order-7, 27-quantity workload) against three oracle steps; errors of each quantity
    relative to the norm of that quantity's change."""
    N = order - 1
    mesh = wl.jittered_periodic_mesh(3, jitter=0.1, seed=17)
    el = mesh.elements
    dt = wl.cfl_time_step(el, N)
    att = wl.attenuation(el, dt, seed=19)
    Q0 = wl.random_dofs_viscoelastic(el.rho.size, basis.n_basis(N), el, att, seed=20)
    s = solver(yt, el, mesh.conn, dt, att, order, getattr(yt, prec_name))
    s.set_dofs_host(Q0)
    for _ in range(3):
        s.step()
    q = s.get_host()
    s.close()
    Q, _ = oracle_steps(el, mesh.conn, dt, att, Q0, order, steps=3)
    if tol is None:
        tol, tol_el = parity.VE_F32_INC, parity.VE_F32_INC_EL
    elif tol == "tc":
        tol, tol_el = parity.VE_TC_INC, parity.VE_TC_INC_EL
    parity.check(f"ve {prec_name} jittered o{order} 3 steps dQ", q, Q, tol, tol_el, base=Q0)


def test_ve_degenerate_inputs(yt):
    """Zero DOFs stay exactly zero (FP32 and tensor-core forms); a single element whose
    faces are its own neighbours; the unfused pair is refused for 27 quantities."""
    el, conn, dt, att, Q = make_case(40, 4, 560)
    for prec in (yt.YT_F32, yt.YT_BF16X3_F32ACC):
        s = solver(yt, el, conn, dt, att, 4, prec)
        s.set_dofs_host(np.zeros_like(Q))
        s.step()
        assert not np.any(s.get_host()) and not np.any(s.get_host(yt.YT_FIELD_TIME_INTEGRAL))
        with pytest.raises(yt.YtError) as info:
            s.step_local()
        assert info.value.status == 4
        s.close()
    # one element, faces paired 0-3 and 1-2 with itself
    e1 = wl.random_elements(1, seed=561)
    dt1 = wl.cfl_time_step(e1, 4)
    a1 = wl.attenuation(e1, dt1, seed=562)
    Q1 = wl.random_dofs_viscoelastic(1, basis.n_basis(4), e1, a1, seed=563)
    c1 = wl.Connectivity(np.zeros((1, 4), dtype=np.int32), np.array([[3, 2, 1, 0]], dtype=np.int8),
                         np.array([[0, 1, 2, 1]], dtype=np.int8))
    s = solver(yt, e1, c1, dt1, a1, 5, yt.YT_F64)
    s.set_dofs_host(Q1)
    s.step()
    q = s.get_host()
    s.close()
    ref, _ = oracle_steps(e1, c1, dt1, a1, Q1, 5)
    parity.check("ve f64 self neighbour dQ", q, ref, parity.F64_INC, parity.F64_INC, base=Q1)
