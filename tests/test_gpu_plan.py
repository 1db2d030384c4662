"""Parity of the batched executor (yt_execute_batched, through the C ABI) with the oracle:
random Einstein expressions against the brute-force Eq. gentensorop, and the four SeisSol
kernels (Sec. 5.1.1) written as expressions against the direct oracle."""
import numpy as np
import pytest

import workload as wl
from oracle import basis, scheme
from oracle import einsum as es

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def yt():
    import paper_1903_11521_gb300 as yt
    yt.load()
    return yt


def to_dev(arr, dtype):
    import torch
    from paper_1903_11521_gb300 import element_major
    return torch.from_numpy(element_major(arr).astype(dtype)).cuda()


def from_dev(t, shape):
    from paper_1903_11521_gb300 import from_element_major
    return from_element_major(t.cpu().numpy().astype(np.float64), shape)


def run(yt, expr, consts, per_elem, out_name, out_shape, E, precision=0, out_init=None):
    import torch
    dtype = np.float64 if precision == 0 else np.float32
    tensors = []
    dev = {}
    for name, arr in per_elem.items():
        tensors.append((name, arr.shape[1:], None, None))
        dev[name] = to_dev(arr, dtype)
    init = out_init if out_init is not None else np.full((E,) + out_shape, 7.0)
    tensors.append((out_name, out_shape, None, None))
    dev[out_name] = to_dev(init, dtype)
    for name, (val, pat) in consts.items():
        tensors.append((name, val.shape, pat, val))
    plan = yt.Plan(expr, tensors, precision=precision)
    plan.execute(dev, E)
    torch.cuda.synchronize()
    return from_dev(dev[out_name], out_shape), plan


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("E", [1, 37])
def test_random_expressions(yt, seed, E):
    rng = np.random.default_rng(seed)
    sizes = {'i': 3, 'j': 2, 'k': 4, 'l': 3, 'm': 2}
    A = rng.standard_normal((sizes['i'], sizes['k'])) * (rng.random((3, 4)) < 0.7)
    Bp = rng.standard_normal((E, sizes['k'], sizes['j'], sizes['l']))
    w = rng.standard_normal((E, sizes['l'], sizes['m']))
    out, plan = run(yt, "U[imj] = 0.5 * A[ik] * B[kjl] * w[lm]", {'A': (A, None)},
                    {'B': Bp, 'w': w}, 'U', (3, 2, 2), E)
    for e in range(E):
        ref = 0.5 * es.einsum_bruteforce('imj', [('ik', A), ('kjl', Bp[e]), ('lm', w[e])])
        assert np.allclose(out[e], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_accumulate_and_assign(yt):
    rng = np.random.default_rng(5)
    E = 40
    X = rng.standard_normal((E, 4, 3))
    K = rng.standard_normal((5, 4))
    init = rng.standard_normal((E, 5, 3))
    out, _ = run(yt, "Y[ap] += K[ab] * X[bp] + 2.0 * K[ab] * X[bp]", {'K': (K, None)}, {'X': X}, 'Y',
                 (5, 3), E, out_init=init)
    assert np.allclose(out, init + 3.0 * np.einsum('ab,ebp->eap', K, X), rtol=1e-13, atol=1e-12)
    out, _ = run(yt, "Y[ap] = K[ab] * X[bp]", {'K': (K, None)}, {'X': X}, 'Y', (5, 3), E, out_init=init)
    assert np.allclose(out, np.einsum('ab,ebp->eap', K, X), rtol=1e-13, atol=1e-12)
    # transposed copy (single factor)
    out, _ = run(yt, "Z[pb] = X[bp]", {}, {'X': X}, 'Z', (3, 4), E)
    assert np.array_equal(out, X.transpose(0, 2, 1))


def _seissol_inputs(order, E):
    N = order - 1
    el = wl.random_elements(E, seed=11)
    conn = wl.random_connectivity(E, seed=12)
    Q = wl.random_dofs(E, basis.n_basis(N), seed=13, scale="impedance", elements=el)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    return N, Q, star, loc, nb, conn


@pytest.mark.parametrize("order", [3, 4])
def test_seissol_kernels_as_expressions(yt, order):
    E = 45
    N, Q, star, loc, nb, conn = _seissol_inputs(order, E)
    m = basis.float_matrices(N)
    B, Bt = basis.n_basis(N), basis.n_face_basis(N)
    As = {f"A{x}": star[:, x] for x in range(3)}
    # derivative (Eq. seissol:derivative)
    consts = {f"K{x}": (m['Ktilde'][x], None) for x in range(3)}
    out, plan = run(yt, "D[kp] = K0[kl]*Q[lq]*A0[pq] + K1[kl]*Q[lq]*A1[pq] + K2[kl]*Q[lq]*A2[pq]",
                    consts, {'Q': Q, **As}, 'D', (B, 9), E)
    ref = sum(np.matmul(np.matmul(m['Ktilde'][x], Q), np.swapaxes(star[:, x], -1, -2)) for x in range(3))
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    assert plan.stats()['n_terms'] == 3
    # volume (Eq. seissol:correction_local, first part)
    consts = {f"K{x}": (m['Khat'][x], None) for x in range(3)}
    out, _ = run(yt, "V[kp] += K0[kl]*I[lq]*A0[pq] + K1[kl]*I[lq]*A1[pq] + K2[kl]*I[lq]*A2[pq]",
                 consts, {'I': Q, **As}, 'V', (B, 9), E, out_init=Q)
    ref = Q + sum(np.matmul(np.matmul(m['Khat'][x], Q), np.swapaxes(star[:, x], -1, -2)) for x in range(3))
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    # local flux of face 2 (Rhat R^T)
    s = 2
    consts = {'Rh': (m['Rhat'][s], None), 'R': (m['R'][s], None)}
    out, _ = run(yt, "F[kp] = Rh[km] * R[lm] * I[lq] * Al[pq]", consts, {'I': Q, 'Al': loc[:, s]},
                 'F', (B, 9), E)
    ref = np.matmul(np.matmul(m['FmHat'][s], Q), np.swapaxes(loc[:, s], -1, -2))
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    # neighbour flux of face 1 for fixed (j, h) = (3, 2), neighbour DOFs gathered
    j, h = 3, 2
    Inb = Q[conn.neighbours[:, 1]]
    consts = {'Rh': (m['Rhat'][1], None), 'f': (m['f'][h], None), 'R': (m['R'][j], None)}
    out, plan = run(yt, "G[kp] = Rh[km] * f[mn] * R[ln] * J[lq] * An[pq]", consts,
                    {'J': Inb, 'An': nb[:, 1]}, 'G', (B, 9), E)
    ref = np.matmul(np.matmul(m['FpHat'][1, j, h], Inb), np.swapaxes(nb[:, 1], -1, -2))
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_single_precision_plan(yt):
    E = 64
    N, Q, star, loc, nb, conn = _seissol_inputs(4, E)
    m = basis.float_matrices(N)
    B = basis.n_basis(N)
    out, _ = run(yt, "V[kp] = K0[kl]*I[lq]*A0[pq]", {'K0': (m['Khat'][0], None)},
                 {'I': Q, 'A0': star[:, 0]}, 'V', (B, 9), E, precision=1)
    ref = np.matmul(np.matmul(m['Khat'][0], Q), np.swapaxes(star[:, 0], -1, -2))
    assert np.linalg.norm(out - ref) <= 2e-6 * np.linalg.norm(ref)


def test_many_elements_sampled(yt):
    """100,003 elements (several grid-stride passes per warp slot), sampled checks."""
    rng = np.random.default_rng(9)
    E = 100_003
    K = rng.standard_normal((6, 5))
    X = rng.standard_normal((E, 5, 4))
    out, _ = run(yt, "Y[ap] = K[ab] * X[bp]", {'K': (K, None)}, {'X': X}, 'Y', (6, 4), E)
    idx = rng.integers(0, E, 200).tolist() + [0, E - 1]
    ref = np.einsum('ab,ebp->eap', K, X[idx])
    assert np.allclose(out[idx], ref, rtol=1e-13, atol=1e-12)


def test_zero_elements_is_a_no_op(yt):
    import torch
    plan = yt.Plan("Y[ap] = K[ab] * X[bp]", [('K', (2, 2), None, np.eye(2)), ('X', (2, 2), None, None),
                                             ('Y', (2, 2), None, None)])
    y = torch.full((4,), 3.0, dtype=torch.float64, device='cuda')
    plan.execute({'X': y, 'Y': y}, 0)
    torch.cuda.synchronize()
    assert (y == 3.0).all()


def test_lina_kernels_as_expressions(yt):
    """The LinA (ADER-DG-SEM, 3D linearised acoustics, Sec. 5.2) kernels as expressions:
    tensor-product CK derivative, volume, boundary-node extraction and the flux of one
    pair of sides, with global 1D matrices, sparse 4 x 4 Jacobians (constant material on a
    uniform mesh) and per-element DOF tensors, against the brute-force Eq. gentensorop."""
    rng = np.random.default_rng(21)
    n, E = 4, 11                                   # N + 1 nodes per direction
    Kt, Kh = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    # acoustic Jacobians, q = (pressure, u, v, w): A couples p-u, B p-v, C p-w
    jac = []
    for d in range(3):
        M = np.zeros((4, 4))
        M[0, d + 1] = rng.uniform(1, 2)
        M[d + 1, 0] = rng.uniform(1, 2)
        jac.append(M)
    As, Bs, Cs = jac
    Ap, Am = rng.standard_normal((4, 4)), rng.standard_normal((4, 4))
    Fs = np.zeros(n)
    Fs[n - 1] = 1.0                                # F^sigma_i = delta_iN (right/top/front)
    Fh = rng.standard_normal(n)
    D0 = rng.standard_normal((E, n, n, n, 4))
    consts = {'Kt': (Kt, None), 'As': (As, As != 0), 'Bs': (Bs, Bs != 0), 'Cs': (Cs, Cs != 0)}
    out, plan = run(yt, "D1[xyzp] = Kt[xl] * D0[lyzq] * As[pq] + Kt[ym] * D0[xmzq] * Bs[pq]"
                        " + Kt[zn] * D0[xynq] * Cs[pq]", consts, {'D0': D0}, 'D1', (n, n, n, 4), E)
    assert plan.stats()['n_terms'] == 3
    for e in (0, E - 1):
        ref = (es.einsum_bruteforce('xyzp', [('xl', Kt), ('lyzq', D0[e]), ('pq', As)]) +
               es.einsum_bruteforce('xyzp', [('ym', Kt), ('xmzq', D0[e]), ('pq', Bs)]) +
               es.einsum_bruteforce('xyzp', [('zn', Kt), ('xynq', D0[e]), ('pq', Cs)]))
        assert np.allclose(out[e], ref, rtol=1e-13, atol=1e-12 * np.abs(ref).max())
    # volume: Q* = Q + Khat terms on the time integral
    I = rng.standard_normal((E, n, n, n, 4))
    Q = rng.standard_normal((E, n, n, n, 4))
    consts = {'Kh': (Kh, None), 'As': (As, As != 0), 'Bs': (Bs, Bs != 0), 'Cs': (Cs, Cs != 0)}
    out, _ = run(yt, "Qs[xyzp] += Kh[xl] * I[lyzq] * As[pq] + Kh[ym] * I[xmzq] * Bs[pq]"
                     " + Kh[zn] * I[xynq] * Cs[pq]", consts, {'I': I}, 'Qs', (n, n, n, 4), E, out_init=Q)
    ref = Q + (np.einsum('xl,elyzq,pq->exyzp', Kh, I, As) + np.einsum('ym,exmzq,pq->exyzp', Kh, I, Bs)
               + np.einsum('zn,exynq,pq->exyzp', Kh, I, Cs))
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-12 * np.abs(ref).max())
    # boundary nodes of one side (a copy expressed as a product with a selection vector)
    out_z, _ = run(yt, "Z[xyp] = F[n] * I[xynp]", {'F': (Fs, Fs != 0)}, {'I': I}, 'Z', (n, n, 4), E)
    assert np.array_equal(out_z, I[:, :, :, n - 1, :])
    # flux of the side pair in z: own boundary nodes with A+, the neighbour's with A-
    Zn = np.roll(out_z, 1, axis=0)                 # neighbour of element e: e - 1
    consts = {'Fh': (Fh, None), 'Ap': (Ap, None), 'Am': (Am, None)}
    out, _ = run(yt, "Qn[xyzp] += Fh[z] * Z[xyq] * Ap[pq] + Fh[z] * Zn[xyq] * Am[pq]", consts,
                 {'Z': out_z, 'Zn': Zn}, 'Qn', (n, n, n, 4), E, out_init=Q)
    for e in (0, 5):
        ref = Q[e] + es.einsum_bruteforce('xyzp', [('z', Fh), ('xyq', out_z[e]), ('pq', Ap)]) + \
            es.einsum_bruteforce('xyzp', [('z', Fh), ('xyq', Zn[e]), ('pq', Am)])
        assert np.allclose(out[e], ref, rtol=1e-13, atol=1e-12 * np.abs(ref).max())


def _viscoelastic_shaped(star9, n_mech, rng):
    """27-quantity (n_mech = 3) star and source matrices with the block structure of an
    anelastic extension: the elastic 9 x 9 block (from the elastic setup), rows of 6 memory
    variables per mechanism driven by the three velocities (the stress-velocity pattern,
    synthetic scale per mechanism), and a source coupling memory variables to themselves
    (decay) and to the stresses.  Values synthetic; the paper gives no equations for this
    rheology, so only the contraction structure is exercised."""
    E = star9.shape[0]
    P = 9 + 6 * n_mech
    A = np.zeros((E, 3, P, P))
    A[:, :, :9, :9] = star9
    Esrc = np.zeros((E, P, P))
    for m in range(n_mech):
        r = 9 + 6 * m
        A[:, :, r:r + 6, 6:9] = star9[:, :, 0:6, 6:9] * rng.uniform(0.1, 1.0, (E, 1, 1, 1))
        w = rng.uniform(0.5, 2.0, E)
        Esrc[:, r:r + 6, r:r + 6] = -w[:, None, None] * np.eye(6)
        Esrc[:, 0:6, r:r + 6] = rng.uniform(-1.0, 1.0, (E, 6, 6)) * np.eye(6)
    return A, Esrc


@pytest.mark.parametrize("precision, tol", [(0, 1e-12), (1, 5e-6)])
def test_viscoelastic_shaped_kernels_as_expressions(yt, precision, tol):
    """Derivative with a reactive source term, volume and local flux of a 27-quantity
    system, block-sparse per-element matrices passed with their patterns, order 6, against
    the plain definition (matrix products in FP64) and, for two elements, Eq. gentensorop.
    FP32 bound 5e-6: binary32 rounding (6e-8) over sums of up to 56 + 27 products."""
    rng = np.random.default_rng(27)
    order, E = 6, 40
    N, _, star, loc, _, _ = _seissol_inputs(order, E)
    m = basis.float_matrices(N)
    B, P = basis.n_basis(N), 27
    A, Esrc = _viscoelastic_shaped(star, 3, rng)
    D = rng.standard_normal((E, B, P))
    per = {'D': D, 'Es': Esrc, **{f"A{x}": A[:, x] for x in range(3)}}
    consts = {f"K{x}": (m['Ktilde'][x], None) for x in range(3)}
    expr = "D1[kp] = K0[kl]*D[lq]*A0[pq] + K1[kl]*D[lq]*A1[pq] + K2[kl]*D[lq]*A2[pq] + D[kq]*Es[pq]"
    # per-element block patterns: the executor multiplies only their non-zeros
    tensors_pat = {f"A{x}": (A[:, x] != 0).any(axis=0) for x in range(3)}
    tensors_pat['Es'] = (Esrc != 0).any(axis=0)
    out, plan = _run_with_patterns(yt, expr, consts, per, tensors_pat, 'D1', (B, P), E, precision)
    ref = sum(np.matmul(np.matmul(m['Ktilde'][x], D), np.swapaxes(A[:, x], -1, -2)) for x in range(3)) \
        + np.matmul(D, np.swapaxes(Esrc, -1, -2))
    assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref)
    assert plan.stats()['n_terms'] == 4
    if precision == 0:
        for e in (0, E - 1):
            bf = sum(es.einsum_bruteforce('kp', [('kl', m['Ktilde'][x]), ('lq', D[e]), ('pq', A[e, x])])
                     for x in range(3)) + es.einsum_bruteforce('kp', [('kq', D[e]), ('pq', Esrc[e])])
            assert np.allclose(out[e], bf, rtol=1e-13, atol=1e-12 * np.abs(bf).max())
    # volume with the 27 x 27 stars
    consts = {f"K{x}": (m['Khat'][x], None) for x in range(3)}
    Q = rng.standard_normal((E, B, P))
    per = {'I': D, **{f"A{x}": A[:, x] for x in range(3)}}
    out, _ = _run_with_patterns(yt, "V[kp] += K0[kl]*I[lq]*A0[pq] + K1[kl]*I[lq]*A1[pq] + K2[kl]*I[lq]*A2[pq]",
                                consts, per, tensors_pat, 'V', (B, P), E, precision, out_init=Q)
    ref = Q + sum(np.matmul(np.matmul(m['Khat'][x], D), np.swapaxes(A[:, x], -1, -2)) for x in range(3))
    assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref)
    # local flux of face 0 with a dense 27 x 27 flux solver
    Al = rng.standard_normal((E, P, P))
    consts = {'Rh': (m['Rhat'][0], None), 'R': (m['R'][0], None)}
    out, _ = _run_with_patterns(yt, "F[kp] = Rh[km] * R[lm] * I[lq] * Al[pq]", consts,
                                {'I': D, 'Al': Al}, {}, 'F', (B, P), E, precision)
    ref = np.matmul(np.matmul(m['FmHat'][0], D), np.swapaxes(Al, -1, -2))
    assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref)


def _run_with_patterns(yt, expr, consts, per_elem, patterns, out_name, out_shape, E, precision,
                       out_init=None):
    """As run(), with non-zero patterns for per-element tensors."""
    import torch
    dtype = np.float64 if precision == 0 else np.float32
    tensors, dev = [], {}
    for name, arr in per_elem.items():
        tensors.append((name, arr.shape[1:], patterns.get(name), None))
        dev[name] = to_dev(arr, dtype)
    init = out_init if out_init is not None else np.full((E,) + out_shape, 7.0)
    tensors.append((out_name, out_shape, None, None))
    dev[out_name] = to_dev(init, dtype)
    for name, (val, pat) in consts.items():
        tensors.append((name, val.shape, pat, val))
    plan = yt.Plan(expr, tensors, precision=precision)
    plan.execute(dev, E)
    torch.cuda.synchronize()
    return from_dev(dev[out_name], out_shape), plan


@pytest.mark.parametrize("S", [2, 4, 8])
def test_fused_simulation_chain_both_executor_kernels(yt, S):
    """The neighbour-flux chain of one face with S fused simulations at order 6, against
    the plain definition (matrix products): with 2 and 4 simulations the temporaries of
    four warps fit in 96 KB of shared memory (element-per-warp kernel; 4: above the 48 KB
    that need the opt-in attribute), with 8 they do not (lane-per-element kernel,
    temporaries in global scratch)."""
    rng = np.random.default_rng(40 + S)
    order, E = 6, 37
    N = order - 1
    m = basis.float_matrices(N)
    B, Bt = basis.n_basis(N), basis.n_face_basis(N)
    J = rng.standard_normal((E, B, 9, S))
    A = rng.standard_normal((E, 9, 9))
    consts = {'Rh': (m['Rhat'][1], m['Rhat'][1] != 0), 'f': (m['f'][2], m['f'][2] != 0),
              'R': (m['R'][3], m['R'][3] != 0)}
    out, plan = run(yt, "G[kps] = Rh[km] * f[mn] * R[ln] * J[lqs] * An[pq]", consts,
                    {'J': J, 'An': A}, 'G', (B, 9, S), E)
    F = m['Rhat'][1] @ m['f'][2] @ m['R'][3].T
    ref = np.einsum('kl,elqs,epq->ekps', F, J, A)
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
