"""Host-side pieces of bench.py (no device work): its command line, the timed CPU
baseline (the oracle step over a sample, chunked over a process pool) and the
diagnostics the structured-mesh form reports (mass diagonal, elastic energy)."""
import sys

import numpy as np
import pytest

import bench
import workload as wl
from oracle import basis, scheme
from paper_1903_11521_gb300 import _lib


def _parse(argv):
    old = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        return bench.parse()
    finally:
        sys.argv = old


@pytest.mark.parametrize("argv", [
    [],
    ["--gpus", "2", "--steps", "3", "--warmup", "3"],
    ["--impl", "reference", "--steps", "2", "--warmup", "3"],
    ["--order", "7", "--precision", "bf16x3", "--steps", "5", "--no-e2e", "--no-cpu-baseline", "--no-forms"],
    ["--order", "7", "--precision", "f32", "--elements", "40000"],
    ["--form", "viscoelastic", "--form-n", "14", "--form-steps", "1"],
    ["--form", "structured"], ["--form", "serving"], ["--form", "executor"], ["--form", "local_update"],
])
def test_command_lines_parse(argv):
    a = _parse(argv)
    assert a.steps >= 1 and a.warmup >= 0


def test_default_run_is_the_headline_workload():
    a = _parse([])
    assert (a.gpus, a.order, a.elements, a.precision, a.impl) == (1, 6, 1_000_000, "f64", "ours")
    assert a.warmup >= 3
    cfg = bench.workload_config(a)
    assert "1000000 tets" in cfg["workload"] and "order 6" in cfg["workload"]
    assert "exceeds the 129 MB L2" in cfg["l2"]


def _ader_step_reference(n, order):
    N = order - 1
    el = wl.random_elements(n)
    conn = wl.random_connectivity(n)
    Q = wl.random_dofs(n, basis.n_basis(N), elements=el)
    dt = wl.cfl_time_step(el, N)
    star, loc, nb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
    ref, _ = scheme.ader_step(Q, star, loc, nb, conn.neighbours, conn.faces, conn.orient, dt, N)
    return ref


def test_cpu_baseline_step_is_the_oracle_step():
    """The timed CPU baseline splits the elements over pool workers and hands each chunk
    the time integrals of its neighbours; the result equals one unsplit oracle step."""
    n, order = 96, 3
    runner = bench.OracleStep(n, order, workers=3)
    try:
        got = runner.step()
    finally:
        runner.close()
    np.testing.assert_array_equal(got.shape, (n, basis.n_basis(order - 1), 9))
    ref = _ader_step_reference(n, order)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("order", [2, 4, 7])
def test_mass_diagonal_is_the_reference_mass(order):
    import paper_1903_11521_gb300 as yt
    _lib.load(build_if_missing=True)
    M = basis.float_matrices(order - 1)["M"]
    np.testing.assert_allclose(bench.mass_diagonal(yt, order), np.diag(M), rtol=1e-13, atol=0)


def _collapsed_rule(n):
    """Gauss rule on the reference tetrahedron by the collapsed (Duffy) map of the unit
    cube, n Gauss-Legendre points per direction: exact for degree <= 2n - 3."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    u, v, t = np.meshgrid(x, x, x, indexing="ij")
    wu, wv, wt = np.meshgrid(w, w, w, indexing="ij")
    zeta = t
    eta = v * (1.0 - t)
    xi = u * (1.0 - v) * (1.0 - t)
    wt_all = wu * wv * wt * (1.0 - v) * (1.0 - t) ** 2
    return np.stack([xi.ravel(), eta.ravel(), zeta.ravel()], 1), wt_all.ravel()


def _voigt_stiffness(lam, mu):
    """6 x 6 isotropic stiffness on (exx, eyy, ezz, 2exy, 2eyz, 2exz) -> (sxx, ..., sxz)."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2 * mu
    C[np.arange(3, 6), np.arange(3, 6)] = mu
    return C


def test_elastic_energy_equals_quadrature_of_the_density():
    """1/2 int (rho |v|^2 + sigma : eps) over each physical tetrahedron, by quadrature of
    the DG polynomial and eps from a 6 x 6 solve with the stiffness (not the closed-form
    compliance the bench uses)."""
    order, E = 4, 5
    N = order - 1
    el = wl.random_elements(E, seed=77)
    q = wl.random_dofs(E, basis.n_basis(N), seed=78, scale="impedance", elements=el)
    pts, w = _collapsed_rule(N + 3)
    phi = basis.evaluate_tet_basis(N, pts)                     # (points, B)
    ref = 0.0
    for e in range(E):
        u = phi @ q[e]                                         # (points, 9)
        C = _voigt_stiffness(el.lam[e], el.mu[e])
        eps_v = np.linalg.solve(C, u[:, :6].T).T               # engineering shear strains
        s_dot_e = (u[:, :6] * eps_v).sum(1)
        dens = el.rho[e] * (u[:, 6:9] ** 2).sum(1) + s_dot_e
        ref += 0.5 * abs(np.linalg.det(el.jac[e])) * float((w * dens).sum())
    Mk = np.diag(basis.float_matrices(N)["M"])
    got = bench.elastic_energy(q, el, Mk, chunk=2)
    assert abs(got - ref) <= 1e-11 * abs(ref)


def test_measured_hbm_peak_and_fallback(monkeypatch, tmp_path):
    """The HBM denominator is the measured copy bandwidth of the peaks file when present,
    else the fallback figure."""
    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 6781.8}')
    monkeypatch.setattr(bench, "PEAKS_FILE", str(f))
    assert bench.measured_hbm_gbs() == 6781.8
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_hbm_gbs() == 6800.0


def _digest_tree(root, kernel_text):
    pkg = root / "paper_1903_11521_gb300"
    (pkg / "csrc").mkdir(parents=True)
    (pkg / "_build" / "gen").mkdir(parents=True)
    (pkg / "csrc" / "ader_kernels.cuh").write_text(kernel_text)
    (pkg / "csrc" / "fp_convert.cuh").write_text("int f(int x) { return x; }\n")
    (pkg / "_build" / "gen" / "yt_rows_o5.cuh").write_text("struct R {};\n")
    for v in ("lf", "nf"):
        (pkg / "_build" / "gen" / f"ader_o5_f64_{v}.cu").write_text(f"// unit {v}\nint u_{v};\n")


def test_kernel_source_digest_ignores_comments_only(monkeypatch, tmp_path):
    """The ncu traffic figure is quoted only while the kernel sources hash to the captured
    version: a comment or whitespace edit keeps the digest, a code edit changes it."""
    base = "__global__ void k(double* q) {\n  q[0] += 1.0;  // one\n}\n"
    variants = {
        "base": base,
        "comment": "/* block\ncomment */\n__global__ void k(double* q) {\n    q[0] += 1.0;  // two\n}\n",
        "code": "__global__ void k(double* q) {\n  q[0] += 2.0;  // one\n}\n",
    }
    digests = {}
    for name, text in variants.items():
        root = tmp_path / name
        _digest_tree(root, text)
        monkeypatch.setattr(bench, "ROOT", str(root))
        digests[name] = bench.kernel_source_digest(6, "f64")
    assert digests["base"] == digests["comment"]
    assert digests["base"] != digests["code"]
    # a missing generated unit changes it too (a stale or partial build is not the capture)
    (tmp_path / "base" / "paper_1903_11521_gb300" / "_build" / "gen" / "ader_o5_f64_nf.cu").unlink()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "base"))
    assert bench.kernel_source_digest(6, "f64") != digests["base"]


def test_ncu_traffic_table_is_per_element_of_a_plausible_size():
    """Each captured traffic figure is bytes per element of one launch pair, between the
    algorithmic bytes of the FP64 step (Q, I, face projections, local flux products) and
    a few times that."""
    for digest, per_order in bench.NCU_TRAFFIC_PER_ELEMENT.items():
        assert len(digest) == 16
        for order, per_element in per_order.items():
            B = basis.n_basis(order - 1)
            algorithmic = 9 * B * 8 * 4                # Q read + written, I written + read
            assert algorithmic <= per_element <= 4 * algorithmic, (digest, order, per_element)
