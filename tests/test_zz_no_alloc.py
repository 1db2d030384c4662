"""yt_execute_batched_noalloc: the executor variant for callers that may not allocate
device memory (its temporaries and tables live in fixed arrays inside the library).
Checked through the C ABI against yt_execute_batched on the same inputs, on two calls in
a row, plus the rejection of a plan whose temporaries exceed the fixed scratch.  This file
is collected last so that a stop at the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _plan_and_inputs(seed, E, precision="YT_F64"):
    import torch

    import paper_1903_11521_gb300 as yt
    from oracle import basis
    rng = np.random.default_rng(seed)
    N = 3
    m = basis.float_matrices(N)
    B, Bt = basis.n_basis(N), basis.n_face_basis(N)
    plan = yt.Plan("G[kp] = Rh[km] * f[mn] * R[ln] * J[lq] * An[pq]",
                   [("Rh", (B, Bt), None, m["Rhat"][1]), ("f", (Bt, Bt), None, m["f"][2]),
                    ("R", (B, Bt), None, m["R"][3]), ("J", (B, 9), None, None),
                    ("An", (9, 9), None, None), ("G", (B, 9), None, None)],
                   precision=getattr(yt, precision))
    dtype = np.float64 if precision == "YT_F64" else np.float32
    J = torch.from_numpy(rng.standard_normal((E, 9 * B)).astype(dtype)).cuda()
    A = torch.from_numpy(rng.standard_normal((E, 81)).astype(dtype)).cuda()
    return plan, J, A, B


def _ptrs(*tensors):
    return (C.c_void_p * len(tensors))(*[C.c_void_p(t.data_ptr()) if t is not None else None
                                         for t in tensors])


# the batched path and the allocation-free path differ only in the order of their
# summations: 1e-12 in binary64, 1e-5 in binary32 (a few units of 2^-24 per product of a
# chain of five factors)
@pytest.mark.parametrize("precision, tol", [("YT_F64", 1e-12), ("YT_F32", 1e-5)])
def test_noalloc_matches_batched_twice(precision, tol):
    import torch

    from paper_1903_11521_gb300 import _lib
    lib = _lib.load()
    E = 1000
    plan, J, A, B = _plan_and_inputs(1, E, precision)
    dtype = J.dtype
    ref = torch.zeros((E, 9 * B), dtype=dtype, device="cuda")
    _lib.check(lib.yt_execute_batched(plan.handle, _ptrs(None, None, None, J, A, ref), E, None),
               "yt_execute_batched")
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full((E, 9 * B), float(call + 5), dtype=dtype, device="cuda")
        _lib.check(lib.yt_execute_batched_noalloc(plan.handle, _ptrs(None, None, None, J, A, out), E, None),
                   "yt_execute_batched_noalloc")
        torch.cuda.synchronize()
        err = (out.double() - ref.double()).norm() / ref.double().norm()
        assert err.item() <= tol, (call, err.item())


def test_noalloc_second_plan_after_first():
    """Consecutive calls with different plans see only their own tables."""
    import torch

    import paper_1903_11521_gb300 as yt
    from paper_1903_11521_gb300 import _lib
    lib = _lib.load()
    E = 77
    plan, J, A, B = _plan_and_inputs(2, E)
    K = np.arange(1.0, 1.0 + B * B).reshape(B, B) / (B * B)
    plan2 = yt.Plan("Y[kq] = K[kl] * J[lq]", [("K", (B, B), None, K), ("J", (B, 9), None, None),
                                              ("Y", (B, 9), None, None)])
    out1 = torch.zeros((E, 9 * B), dtype=torch.float64, device="cuda")
    out2 = torch.zeros_like(out1)
    _lib.check(lib.yt_execute_batched_noalloc(plan.handle, _ptrs(None, None, None, J, A, out1), E, None), "noalloc 1")
    _lib.check(lib.yt_execute_batched_noalloc(plan2.handle, _ptrs(None, J, out2), E, None), "noalloc 2")
    torch.cuda.synchronize()
    Jh = J.cpu().numpy().reshape(E, 9, B).transpose(0, 2, 1)
    ref2 = np.einsum("kl,elq->ekq", K, Jh)
    got2 = out2.cpu().numpy().reshape(E, 9, B).transpose(0, 2, 1)
    assert np.allclose(got2, ref2, rtol=1e-12, atol=1e-12)
    ref1 = torch.zeros_like(out1)
    _lib.check(lib.yt_execute_batched(plan.handle, _ptrs(None, None, None, J, A, ref1), E, None), "batched")
    torch.cuda.synchronize()
    assert ((out1 - ref1).norm() / ref1.norm()).item() <= 1e-12


def test_noalloc_rejects_oversize_temporaries():
    import paper_1903_11521_gb300 as yt
    from paper_1903_11521_gb300 import _lib
    lib = _lib.load()
    # one temporary of 40 x 40 x 40 doubles: 64000 entries x 32 lanes x 8 B x 4 warps > 32 MiB
    plan = yt.Plan("Y[ij] = A[ik] * B[kl] * C[lj] * D[ijkl]",
                   [("A", (40, 40), None, None), ("B", (40, 40), None, None),
                    ("C", (40, 40), None, None), ("D", (40, 40, 40, 40), None, None),
                    ("Y", (40, 40), None, None)])
    status = lib.yt_execute_batched_noalloc(plan.handle, (C.c_void_p * 5)(1, 1, 1, 1, 1), 1, None)
    assert status == 4
    assert b"allocation-free scratch" in lib.yt_last_error()
