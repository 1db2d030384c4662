"""The integer-unit binary32 <-> binary64 conversions of the reduced-precision kernels
against the hardware conversions on the device (exhaustive widening, 2^28 narrowings
including ties and specials)."""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu


def test_conversions_match_hardware():
    import paper_1903_11521_gb300 as yt
    lib = yt.load()
    a, b = C.c_int64(-1), C.c_int64(-1)
    assert lib.yt_selftest_conversions(C.byref(a), C.byref(b)) == 0
    assert a.value == 0 and b.value == 0, (a.value, b.value)
