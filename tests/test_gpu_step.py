"""Parity of the CUDA ADER-DG step (through the C ABI) with the FP64 oracle.

Tolerance: relative Frobenius norm per quantity and per element (tests/parity.py; the
paper compares the optimised and the naive kernel by the Frobenius norm of the
difference, Sec. 4.9): 1e-12 for FP64, the bounds of parity.py for the reduced
precisions."""
import numpy as np
import pytest

import parity
import workload as wl
from oracle import basis, planewave, scheme

pytestmark = pytest.mark.gpu
TOL = parity.F64


@pytest.fixture(scope="module")
def yt():
    import paper_1903_11521_gb300 as yt
    yt.load()
    return yt


def rel_per_quantity(a, b):
    num = np.sqrt(((a - b) ** 2).sum(axis=(0, 1)))
    den = np.sqrt((b ** 2).sum(axis=(0, 1)))
    return num / den


def make_case(E, order, scale, seed=1903):
    N = order - 1
    el = wl.random_elements(E, seed=seed)
    conn = wl.random_connectivity(E, seed=seed + 2)
    Q = wl.random_dofs(E, basis.n_basis(N), seed=seed + 1, scale=scale, elements=el)
    dt = wl.cfl_time_step(el, N)
    return el, conn, Q, dt


def run_gpu(yt, el, conn, Q, dt, order, full=True):
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient)
    s.set_dofs_host(Q)
    if full:
        s.step()
    else:
        s.step_local()
    q = s.get_host(yt.YT_FIELD_DOFS)
    i = s.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    s.close()
    return q, i


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("E", [1, 37, 100])
def test_local_step_parity(yt, order, E):
    """K_local alone (derivatives, time integral, volume, local flux) — the O4 / 1000-tet
    local update is this test at larger E."""
    if E == 1:
        E = 2
    el, conn, Q, dt = make_case(E, order, "impedance")
    q_gpu, i_gpu = run_gpu(yt, el, conn, Q, dt, order, full=False)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    _, I = scheme.derivatives_and_time_integral(Q, star, dt, order - 1)
    q_ref = scheme.local_update(Q, I, star, loc, order - 1)
    parity.check(f"f64 local o{order} E{E} I", i_gpu, I, TOL, TOL)
    parity.check(f"f64 local o{order} E{E} Q", q_gpu, q_ref, TOL, TOL)
    parity.check(f"f64 local o{order} E{E} dQ", q_gpu, q_ref, parity.F64_INC, parity.F64_INC, base=Q)


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_full_step_parity(yt, order):
    E = 70
    el, conn, Q, dt = make_case(E, order, "impedance", seed=7)
    q_gpu, i_gpu = run_gpu(yt, el, conn, Q, dt, order, full=True)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    q_ref, I = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient,
                                dt, order - 1)
    parity.check(f"f64 step o{order} I", i_gpu, I, TOL, TOL)
    parity.check(f"f64 step o{order} Q", q_gpu, q_ref, TOL, TOL)
    parity.check(f"f64 step o{order} dQ", q_gpu, q_ref, parity.F64_INC, parity.F64_INC, base=Q)


def test_config1_local_update_unit_dofs(yt):
    """Order 4, 1000 tets, N(0,1) DOFs, one local update."""
    el, conn, Q, dt = make_case(1000, 4, "unit")
    q_gpu, i_gpu = run_gpu(yt, el, conn, Q, dt, 4, full=False)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    _, I = scheme.derivatives_and_time_integral(Q, star, dt, 3)
    q_ref = scheme.local_update(Q, I, star, loc, 3)
    parity.check("f64 config1 I", i_gpu, I, TOL, TOL)
    parity.check("f64 config1 Q", q_gpu, q_ref, TOL, TOL)


@pytest.mark.parametrize("order", [2, 3, 4, 5])
@pytest.mark.parametrize("prec_name", ["YT_F64", "YT_F32"])
def test_small_mesh_local_kernel_equals_tile_kernel(yt, order, prec_name):
    """The local update of a mesh of at most one tile per SM runs on 8-element CTAs
    (k_local_small, orders <= 5); one tile more selects the 32-element kernel.  The local
    update is element-local, so the first elements of the larger mesh must come out
    bitwise as in the smaller mesh (same arithmetic in the same order), with a ragged
    last tile; both against the oracle."""
    import torch
    prec = getattr(yt, prec_name)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    E_small = 32 * sms - 5                       # ragged last tile, tiles = SMs
    E_big = 32 * sms + 40                        # tiles > SMs
    el, conn, Q, dt = make_case(E_big, order, "impedance", seed=33)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    outs = []
    for E in (E_small, E_big):
        s = yt.Solver(order, dt, mat[:E], el.jac[:E], None, None, None, precision=prec)
        s.set_dofs_host(Q[:E])
        s.step_local()
        outs.append((s.get_host()[:E_small], s.get_host(yt.YT_FIELD_TIME_INTEGRAL)[:E_small]))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    sub = np.arange(0, E_small, 97)
    star, loc, nb = scheme.setup_element_matrices(el.rho[sub], el.lam[sub], el.mu[sub], el.jac[sub])
    _, I = scheme.derivatives_and_time_integral(Q[sub], star, dt, order - 1)
    q_ref = scheme.local_update(Q[sub], I, star, loc, order - 1)
    if prec == yt.YT_F64:
        parity.check(f"small-mesh local o{order} f64 I", outs[0][1][sub], I, TOL, TOL)
        parity.check(f"small-mesh local o{order} f64 dQ", outs[0][0][sub], q_ref, parity.F64_INC,
                     parity.F64_INC, base=Q[sub])
    else:
        parity.check(f"small-mesh local o{order} f32 dQ", outs[0][0][sub], q_ref, parity.F32_INC,
                     parity.F32_INC_EL, base=Q[sub])


def test_plane_wave_on_device(yt):
    """Several steps on the periodic mesh: matches the oracle step by step and converges
    to the closed-form plane wave like the oracle does."""
    order, N = 3, 2
    k = 2 * np.pi * np.array([1.0, 1.0, 0.0])
    mesh = wl.periodic_cube_mesh(4)
    el = mesh.elements
    T = 0.03
    steps = int(np.ceil(T / wl.cfl_time_step(el, N, cfl=0.3)))
    dt = T / steps
    Q0 = planewave.project(mesh, N, 0.0, k, 1.0, 2.0, 1.0)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    s = yt.Solver(order, dt, mat, el.jac, mesh.conn.neighbours, mesh.conn.faces, mesh.conn.orient)
    s.set_dofs_host(Q0)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    Q = Q0
    for _ in range(steps):
        s.step()
        Q, _ = scheme.ader_step(Q, star, loc, nb, mesh.conn.neighbours, mesh.conn.faces,
                                mesh.conn.orient, dt, N)
    q_gpu = s.get_host()
    s.close()
    parity.check("f64 plane wave Q", q_gpu, Q, 1e-11, 1e-11)
    err_gpu = planewave.l2_error(mesh, N, q_gpu, T, k, 1.0, 2.0, 1.0)
    err_ora = planewave.l2_error(mesh, N, Q, T, k, 1.0, 2.0, 1.0)
    assert np.allclose(err_gpu, err_ora, rtol=1e-6)
    assert err_gpu[6] < 0.05


def test_deterministic(yt):
    el, conn, Q, dt = make_case(64, 5, "unit", seed=3)
    a, _ = run_gpu(yt, el, conn, Q, dt, 5)
    b, _ = run_gpu(yt, el, conn, Q, dt, 5)
    assert np.array_equal(a, b)


def test_phases_equal_step_and_unfused_path(yt):
    """yt_step == phase 0 + phase 1 (bitwise); the unfused pair yt_step_local +
    yt_step_neighbour agrees within the FP64 tolerance."""
    el, conn, Q, dt = make_case(96, 6, "impedance", seed=21)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    outs = []
    for mode in ("step", "phases", "unfused"):
        s = yt.Solver(6, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient)
        s.set_dofs_host(Q)
        if mode == "step":
            s.step()
        elif mode == "phases":
            s.step_phase(0)
            s.step_phase(1)
        else:
            s.step_local()
            s.step_neighbour()
        outs.append(s.get_host())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    parity.check("f64 unfused vs fused", outs[2], outs[0], TOL, TOL)


@pytest.mark.parametrize("E", [8 * 32 * 3 + 45, 512 * 32 + 77])
@pytest.mark.parametrize("prec_name", ["YT_F64", "YT_F32", "YT_BF16X3_F32ACC"])
def test_step_host_equals_step(yt, prec_name, E):
    """yt_step_host (pipelined copies, up to 16 element chunks, ragged last chunk and tile; 26 and
    515 tiles) gives bitwise the result of set_dofs + yt_step + get on the same solver;
    also in place."""
    import torch
    prec = getattr(yt, prec_name)
    order = 4
    el, conn, Q, dt = make_case(E, order, "impedance", seed=61)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    canon = np.ascontiguousarray(Q.transpose(0, 2, 1))
    s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient, precision=prec)
    s.set_dofs_host(Q)
    s.step()
    ref = s.get_host()
    pin_in = torch.from_numpy(canon.copy()).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    s.step_host_ptr(pin_in.data_ptr(), pin_out.data_ptr())
    torch.cuda.synchronize()
    got = pin_out.numpy().transpose(0, 2, 1)
    assert np.array_equal(got, ref)
    s.step_host_ptr(pin_in.data_ptr(), pin_in.data_ptr())      # in place
    torch.cuda.synchronize()
    assert np.array_equal(pin_in.numpy().transpose(0, 2, 1), ref)
    s.status()
    s.close()


# ------------------------------------------------------------------ precision form (FP32)
F32_TOL_INCREMENT = parity.F32_INC    # relative Frobenius norm of Q_new - Q
F32_TOL_I = parity.F32_I              # of the time integral


def run_gpu_prec(yt, el, conn, Q, dt, order, precision, full=True, steps=1):
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient, precision=precision)
    s.set_dofs_host(Q)
    for _ in range(steps):
        s.step() if full else s.step_local()
    q = s.get_host(yt.YT_FIELD_DOFS)
    i = s.get_host(yt.YT_FIELD_TIME_INTEGRAL)
    s.close()
    return q, i


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_f32_full_step_against_fp64_oracle(yt, order):
    """Bulk contractions in FP32, setup / time-integral accumulation / DOFs in FP64."""
    el, conn, Q, dt = make_case(70, order, "impedance", seed=31)
    q32, i32 = run_gpu_prec(yt, el, conn, Q, dt, order, yt.YT_F32)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    q_ref, I = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient,
                                dt, order - 1)
    parity.check(f"f32 step o{order} I", i32, I, F32_TOL_I, parity.F32_I_EL)
    parity.check(f"f32 step o{order} dQ", q32, q_ref, F32_TOL_INCREMENT, parity.F32_INC_EL, base=Q)


def test_f32_local_step_order7(yt):
    el, conn, Q, dt = make_case(45, 7, "impedance", seed=32)
    q32, i32 = run_gpu_prec(yt, el, conn, Q, dt, 7, yt.YT_F32, full=False)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    _, I = scheme.derivatives_and_time_integral(Q, star, dt, 6)
    q_ref = scheme.local_update(Q, I, star, loc, 6)
    parity.check("f32 local o7 I", i32, I, F32_TOL_I, parity.F32_I_EL)
    parity.check("f32 local o7 dQ", q32, q_ref, F32_TOL_INCREMENT, parity.F32_INC_EL, base=Q)


def test_f32_plane_wave_100_steps(yt):
    """100 steps at order 5 on the periodic mesh: the FP32 form stays within a stated
    bound of the FP64 path (itself equal to the oracle step by step) and its plane-wave
    error equals the FP64 one to 1e-3 relative."""
    order, N = 5, 4
    k = 2 * np.pi * np.array([1.0, 1.0, 0.0])
    mesh = wl.periodic_cube_mesh(3)
    el = mesh.elements
    dt = wl.cfl_time_step(el, N, cfl=0.3)
    T = 100 * dt
    Q0 = planewave.project(mesh, N, 0.0, k, 1.0, 2.0, 1.0)
    q64, _ = run_gpu_prec(yt, el, mesh.conn, Q0, dt, order, yt.YT_F64, steps=100)
    q32, _ = run_gpu_prec(yt, el, mesh.conn, Q0, dt, order, yt.YT_F32, steps=100)
    drift = rel_per_quantity(q32, q64).max()
    print(f"PARITY f32 plane wave 100 steps drift {drift:.3e} (bound 1e-4)")
    assert drift < 1e-4, drift
    e64 = planewave.l2_error(mesh, N, q64, T, k, 1.0, 2.0, 1.0)
    e32 = planewave.l2_error(mesh, N, q32, T, k, 1.0, 2.0, 1.0)
    assert np.allclose(e32, e64, rtol=1e-3)


def test_f32_order7_100_steps_against_oracle(yt):
    """Order 7 (B = 84) in FP32 contractions, 100 steps of the plane wave on the periodic
    mesh against 100 oracle steps.  The wave has quantities of zero exact amplitude
    (sigma_yz, sigma_xz, w) whose norms sit at the discretisation-error level, so the error
    of each quantity is stated relative to the norm of the whole solution (unit material:
    stresses and velocities of one magnitude): bound 5e-6 (measured 6.0e-7), per element
    1.5e-5 (measured 1.6e-6)."""
    order, N = 7, 6
    k = 2 * np.pi * np.array([1.0, 1.0, 0.0])
    mesh = wl.periodic_cube_mesh(3)
    el = mesh.elements
    dt = wl.cfl_time_step(el, N, cfl=0.3)
    Q = planewave.project(mesh, N, 0.0, k, 1.0, 2.0, 1.0)
    q32, _ = run_gpu_prec(yt, el, mesh.conn, Q, dt, order, yt.YT_F32, steps=100)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    for _ in range(100):
        Q, _ = scheme.ader_step(Q, star, loc, nb, mesh.conn.neighbours, mesh.conn.faces,
                                mesh.conn.orient, dt, N)
    per_q = np.sqrt(((q32 - Q) ** 2).sum(axis=(0, 1)))
    err = per_q.max() / np.sqrt((Q ** 2).sum())
    el_err = parity.per_element(q32, Q).max()
    print(f"PARITY f32 o7 100 steps: {err:.3e} of the solution norm (bound 5e-6), per-element "
          f"{el_err:.3e} (bound 1.5e-5); per quantity {np.array2string(rel_per_quantity(q32, Q), precision=2)}")
    assert err < 5e-6
    assert el_err < 1.5e-5


@pytest.mark.parametrize("prec_name, tol_inc", [("YT_F64", parity.F64_INC), ("YT_F32", parity.F32_INC_EL),
                                                ("YT_BF16X3_F32ACC", parity.TC_INC_EL)])
def test_single_element_self_neighbour(yt, prec_name, tol_inc):
    """Degenerate connectivity: one element (one tile of 32 lanes with 31 padding lanes)
    whose four faces are its own neighbours (faces paired 0-3 and 1-2, all orientations):
    the neighbour flux reads the element's own face projections."""
    order, N = 5, 4
    el = wl.random_elements(1, seed=71)
    Q = wl.random_dofs(1, basis.n_basis(N), seed=72, scale="impedance", elements=el)
    dt = wl.cfl_time_step(el, N)
    nbr = np.zeros((1, 4), dtype=np.int32)
    faces = np.array([[3, 2, 1, 0]], dtype=np.int8)
    orient = np.array([[0, 1, 2, 1]], dtype=np.int8)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    s = yt.Solver(order, dt, mat, el.jac, nbr, faces, orient, precision=getattr(yt, prec_name))
    s.set_dofs_host(Q)
    s.step()
    s.status()
    q = s.get_host()
    s.close()
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref, _ = scheme.ader_step(Q, star, loc, nb, nbr, faces, orient, dt, N)
    parity.check(f"{prec_name} self neighbour dQ", q, ref, tol_inc, tol_inc, base=Q)


def test_zero_dofs_stay_zero(yt):
    """The step is linear in Q: zero DOFs give exactly zero, in every precision."""
    el, conn, Q, dt = make_case(64, 4, "unit", seed=73)
    mat = np.stack([el.rho, el.lam, el.mu], axis=1)
    for prec in (yt.YT_F64, yt.YT_F32, yt.YT_BF16X3_F32ACC):
        s = yt.Solver(4, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient, precision=prec)
        s.set_dofs_host(np.zeros_like(Q))
        s.step()
        s.status()
        assert not np.any(s.get_host())
        assert not np.any(s.get_host(yt.YT_FIELD_TIME_INTEGRAL))
        s.close()


@pytest.mark.parametrize("prec_name, order, tol, tol_el", [
    ("YT_F64", 6, 1e-12, 1e-11), ("YT_F64", 7, 1e-12, 1e-11),
    ("YT_F32", 7, 1e-6, 3.5e-6), ("YT_BF16X3_F32ACC", 6, 4e-5, 1e-4), ("YT_BF16X3_F32ACC", 7, 4e-5, 1e-4)])
def test_jittered_structured_mesh_steps(yt, prec_name, order, tol, tol_el):
    """Three steps on the jittered periodic structured mesh (vertices moved by up to 0.1 h,
    the mesh family of the order-7 FP32 workload) against three oracle steps, random
    impedance-scaled DOFs; error per quantity relative to the norm of the whole solution
    change (stated bounds: FP64 1e-12, FP32 1e-6, split-bf16 4e-5, about nine times the
    measured 1.2e-7 and 3.8e-6; per element 1e-11, 3.5e-6, 1e-4)."""
    N = order - 1
    mesh = wl.jittered_periodic_mesh(3, jitter=0.1, seed=17)
    el = mesh.elements
    dt = wl.cfl_time_step(el, N)
    Q0 = wl.random_dofs(el.rho.size, basis.n_basis(N), seed=18, scale="impedance", elements=el)
    q, _ = run_gpu_prec(yt, el, mesh.conn, Q0, dt, order, getattr(yt, prec_name), steps=3)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    Q = Q0
    for _ in range(3):
        Q, _ = scheme.ader_step(Q, star, loc, nb, mesh.conn.neighbours, mesh.conn.faces,
                                mesh.conn.orient, dt, N)
    err = np.sqrt(((q - Q) ** 2).sum(axis=(0, 1))).max() / np.sqrt(((Q - Q0) ** 2).sum())
    el_err = parity.per_element(q - Q0, Q - Q0).max()
    print(f"PARITY {prec_name} jittered o{order} 3 steps: {err:.3e} (bound {tol:.1e}), "
          f"per-element {el_err:.3e} (bound {tol_el:.1e})")
    assert err < tol, err
    assert el_err < tol_el, el_err


def _nonzero_flops(order):
    """Non-zero flops per element of the two step kernels in the convention of Sec. 4.9
    (a sum of n products: 2n - 1 flops assigned, 2n added to an existing value; a scaling:
    1), counted here from the oracle's matrices: derivatives restricted to the staircase,
    volume, face projections, 9 x 9 mixing with the 24-non-zero star matrices, flux
    solvers, block-diagonal f^h, lifting of both flux terms."""
    N = order - 1
    m = basis.float_matrices(N)
    B, BT = basis.n_basis(N), basis.n_face_basis(N)
    nd = lambda d: (N - d + 3) * (N - d + 2) * (N - d + 1) // 6   # noqa: E731
    star_nnz = 24

    def assigned(M):
        n = (M != 0).sum(axis=1)
        return 9 * int(np.where(n > 0, 2 * n - 1, 0).sum())

    local = 9 * B
    for d in range(N):
        for x in range(3):
            local += assigned(m['Ktilde'][x][:nd(d + 1), :nd(d)])
        local += nd(d + 1) * ((6 * star_nnz - 9) + 2 * 9)
    for x in range(3):
        local += assigned(m['Khat'][x])
    local += B * 6 * star_nnz
    neigh = 0
    for s in range(4):
        local += assigned(m['R'][s].T) + BT * 9 * 17
        blocks = sum((d + 1) * (2 * (d + 1) - 1) for d in range(N + 1))
        neigh += 9 * blocks + BT * 9 * 18 + 9 * 2 * int((m['Rhat'][s] != 0).sum())
    return local, neigh


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_flop_counts_match_pattern_count(yt, order):
    """The flops the library reports (used for every roofline fraction) equal an
    independent count from the oracle's sparsity patterns."""
    el, conn, Q, dt = make_case(40, order, "unit")
    s = yt.Solver(order, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, conn.neighbours,
                  conn.faces, conn.orient)
    st = s.stats()
    s.close()
    local, neigh = _nonzero_flops(order)
    assert st['local_flops'] == local
    assert st['neighbour_flops'] == neigh
