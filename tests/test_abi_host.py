"""Host-side checks of the C ABI library (no device work): it loads, exports every symbol
of include/yateto_gb300.h, validates arguments, and its reference matrices equal the
oracle's exact ones."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import basis
from paper_1903_11521_gb300 import _lib, reference_matrix

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load(build_if_missing=True)


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "yateto_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(yt_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_status_strings_and_version(lib):
    assert lib.yt_status_string(0) == b"YT_OK"
    for s in range(1, 8):
        assert lib.yt_status_string(s).startswith(b"YT_ERR_")
    assert b"sm_103a" in lib.yt_version()


def test_invalid_arguments_rejected_without_device(lib):
    out = C.c_void_p()
    assert lib.yt_solver_create(None, None, None, C.byref(out)) == 1
    assert b"null" in lib.yt_last_error()
    mesh = _lib.MeshDesc(n_elements=0)
    sch = _lib.SchemeDesc(order=4, dt=1e-3, precision=0, flags=0)
    assert lib.yt_solver_create(C.byref(mesh), C.byref(sch), None, C.byref(out)) == 1
    n = C.c_int64()
    assert lib.yt_reference_matrix(9, b"M", None, C.byref(n)) == 1
    assert lib.yt_reference_matrix(4, b"nope", None, C.byref(n)) == 1
    assert lib.yt_step(None, None) == 1


def _create_status(lib, E=4, order=4, dt=1e-3, precision=0, flags=0, quantities=0, neighbours=True,
                   attenuation=False, n_halo=0):
    """Status of yt_solver_create for a descriptor; every case below is rejected before any
    device work (the argument checks come first), so no GPU is needed."""
    n = min(E, 16)             # arrays of the cases that pass the count check; never read
    mat = np.ones((n, 3))
    jac = np.tile(np.eye(3).ravel(), (n, 1))
    nb = np.zeros((n, 4), dtype=np.int32)
    fj = np.zeros((n, 4), dtype=np.int8)
    att = np.ones((n, 9))
    mesh = _lib.MeshDesc(n_elements=E, material=mat.ctypes.data_as(C.POINTER(C.c_double)),
                         jacobian=jac.ctypes.data_as(C.POINTER(C.c_double)), n_halo=n_halo)
    if neighbours:
        mesh.neighbours = nb.ctypes.data_as(C.POINTER(C.c_int32))
        mesh.faces = fj.ctypes.data_as(C.POINTER(C.c_int8))
        mesh.orient = fj.ctypes.data_as(C.POINTER(C.c_int8))
    if attenuation:
        mesh.attenuation = att.ctypes.data_as(C.POINTER(C.c_double))
    sch = _lib.SchemeDesc(order=order, dt=dt, precision=precision, flags=flags, quantities=quantities)
    out = C.c_void_p()
    return lib.yt_solver_create(C.byref(mesh), C.byref(sch), None, C.byref(out))


@pytest.mark.parametrize("case, status", [
    (dict(E=1 << 24), 4),                                  # element index beyond the 24-bit packing
    (dict(order=1), 1), (dict(order=8), 1),                # orders 2..7
    (dict(dt=0.0), 1), (dict(dt=float("nan")), 1),
    (dict(precision=7), 4),
    (dict(flags=1), 1),                                    # diagnostics flag without the tensor cores
    (dict(flags=2, precision=2), 1),                       # unknown flag
    (dict(quantities=10), 1),
    (dict(attenuation=True), 1),                           # attenuation on a 9-quantity solver
    (dict(quantities=27), 1),                              # 27 quantities without attenuation
    (dict(quantities=27, attenuation=True, neighbours=False), 1),
    (dict(n_halo=-1), 1), (dict(n_halo=1 << 26), 1),
    (dict(n_halo=8, precision=2), 4),                      # partitioned tensor-core solves
    (dict(n_halo=8, quantities=27, attenuation=True), 4),  # partitioned 27-quantity solves
])
def test_solver_descriptor_limits_rejected_without_device(lib, case, status):
    assert _create_status(lib, **case) == status, lib.yt_last_error()


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_reference_matrices_match_oracle(order):
    N = order - 1
    ex = basis.float_matrices(N)
    B, Bt = basis.n_basis(N), basis.n_face_basis(N)
    ours = {
        "M": reference_matrix(order, "M"),
        "Khat": reference_matrix(order, "Khat").reshape(3, B, B).transpose(0, 2, 1),
        "Ktilde": reference_matrix(order, "Ktilde").reshape(3, B, B).transpose(0, 2, 1),
        "R": reference_matrix(order, "R").reshape(4, Bt, B).transpose(0, 2, 1),
        "Rhat": reference_matrix(order, "Rhat").reshape(4, Bt, B).transpose(0, 2, 1),
        "f": reference_matrix(order, "f").reshape(3, Bt, Bt).transpose(0, 2, 1),
    }
    assert np.allclose(ours["M"], np.diag(ex["M"]), rtol=1e-14)
    for key in ("Khat", "Ktilde", "R", "Rhat", "f"):
        a, b = ours[key], ex[key]
        assert np.array_equal(a != 0, b != 0), key          # identical sparsity patterns
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-13 * scale, key
