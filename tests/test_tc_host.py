"""Host side of the tensor-core form (no GPU): the split-bf16 global-matrix operands the
library builds for k_local_tc / k_neigh_tc, decoded from their canonical core-matrix
layout and checked against the oracle's matrices: every entry reproduced by hi + lo to
the two-term bf16 split's accuracy, structural zeros and padding exactly zero, each pass
holding the restriction the kernels use (derivative staircase, the volume matrix's
non-zero columns, the four faces' projections stacked, the four liftings stacked)."""
import ctypes as C

import numpy as np
import pytest

from oracle import basis


def up8(x):
    return (x + 7) // 8 * 8


def up16(x):
    return (x + 15) // 16 * 16


def nd(N, d):
    n = N - d
    return (n + 3) * (n + 2) * (n + 1) // 6


def decode(buf, off, n_rows, kp):
    """(hi, lo) float arrays n_rows x kp of the pass at byte offset `off`."""
    out = []
    for part in range(2):
        base = off + part * n_rows * kp * 2
        r = np.arange(n_rows)[:, None]
        k = np.arange(kp)[None, :]
        byte = base + (r // 8) * (kp * 16) + (k // 8) * 128 + (r % 8) * 16 + (k % 8) * 2
        raw = buf[byte] .astype(np.uint32) | (buf[byte + 1].astype(np.uint32) << 8)
        out.append((raw << 16).view(np.float32).astype(np.float64))
    return out


def blob(lib, order, kernel):
    n = C.c_int64()
    assert lib.yt_tc_operands(order, kernel, None, C.byref(n)) == 0
    buf = np.zeros(n.value, dtype=np.uint8)
    assert lib.yt_tc_operands(order, kernel, buf.ctypes.data, C.byref(n)) == 0
    return buf


def check_pass(hi, lo, expect):
    """expect: dense n_rows x kp matrix (zeros where the pass has none)."""
    got = hi + lo
    scale = np.abs(expect)
    assert np.all((expect == 0) == (hi == 0)), "pattern"
    assert np.all(lo[expect == 0] == 0)
    # two-term split: |x - hi - lo| <= 2^-16 |x| (each part rounded to nearest)
    assert np.all(np.abs(got - expect) <= 2.0 ** -16 * scale)


@pytest.fixture(scope="module")
def lib():
    import paper_1903_11521_gb300 as yt
    return yt.load()


def derivative_passes(N):
    """(delta, first output row, rows) of every derivative pass: one per derivative, the
    first split into rows [0, 32) and [32, C(N+2,3)) when its three directions would need
    more than 160 accumulator columns (order 7)."""
    if 3 * up8(nd(N, 1)) > 160:
        return [(0, 0, 32), (0, 32, nd(N, 1) - 32)] + [(d, 0, nd(N, d + 1)) for d in range(1, N)]
    return [(d, 0, nd(N, d + 1)) for d in range(N)]


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_local_operands(lib, order):
    N = order - 1
    m = basis.float_matrices(N)
    B, BT = basis.n_basis(N), basis.n_face_basis(N)
    BT8 = up8(BT)
    buf = blob(lib, order, 0)
    off = 0
    # derivative passes
    passes = derivative_passes(N)
    assert (len(passes) == N + 1) == (order == 7)
    for d, row0, R in passes:
        nin = nd(N, d)
        r8 = up8(R)
        npass, kp = up16(3 * r8), up16(nin)
        assert npass <= 160
        exp = np.zeros((npass, kp))
        for x in range(3):
            exp[x * r8:x * r8 + R, :nin] = m["Ktilde"][x][row0:row0 + R, :nin]
        hi, lo = decode(buf, off, npass, kp)
        check_pass(hi, lo, exp)
        off += 2 * npass * kp * 2
    # volume passes: rows in chunks, columns beyond C(N+2,3) are zero in Khat
    nv = 1
    while up16(3 * up8((B + nv - 1) // nv)) > 160:
        nv += 1
    vr = up8((B + nv - 1) // nv)
    ni = nd(N, 1)
    assert np.all(m["Khat"][:, :, ni:] == 0)
    for v in range(nv):
        k0, rows = v * vr, min(vr, B - v * vr)
        r8 = up8(rows)
        npass, kp = up16(3 * r8), up16(ni)
        exp = np.zeros((npass, kp))
        for x in range(3):
            exp[x * r8:x * r8 + rows, :ni] = m["Khat"][x][k0:k0 + rows, :ni]
        hi, lo = decode(buf, off, npass, kp)
        check_pass(hi, lo, exp)
        off += 2 * npass * kp * 2
    # face projections: column s * BT8 + m, K = l
    npass, kp = up16(4 * BT8), up16(B)
    exp = np.zeros((npass, kp))
    for s in range(4):
        exp[s * BT8:s * BT8 + BT, :B] = m["R"][s].T
    hi, lo = decode(buf, off, npass, kp)
    check_pass(hi, lo, exp)
    off += 2 * npass * kp * 2
    assert off == buf.size


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_neighbour_operands(lib, order):
    N = order - 1
    m = basis.float_matrices(N)
    B, BT = basis.n_basis(N), basis.n_face_basis(N)
    BT8 = up8(BT)
    buf = blob(lib, order, 1)
    npass, kp = up16(B), up16(4 * BT8)
    exp = np.zeros((npass, kp))
    for s in range(4):
        exp[:B, s * BT8:s * BT8 + BT] = m["Rhat"][s]
    hi, lo = decode(buf, 0, npass, kp)
    check_pass(hi, lo, exp)
    assert buf.size == 2 * npass * kp * 2


def test_operands_rejected_out_of_range(lib):
    n = C.c_int64()
    assert lib.yt_tc_operands(8, 0, None, C.byref(n)) == 4     # YT_ERR_UNSUPPORTED
    assert lib.yt_tc_operands(4, 2, None, C.byref(n)) == 1     # YT_ERR_INVALID
