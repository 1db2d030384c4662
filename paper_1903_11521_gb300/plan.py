"""Python view of the planner / batched executor of the C ABI (marshalling only)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from .solver import _stream_handle


class Plan:
    """Plan of an Einstein-notation assignment.

    tensors: list of (name, shape, pattern or None, values or None); a tensor with values
    is a global constant, the others are per-element tensors passed to execute()."""

    def __init__(self, expr: str, tensors, precision=_lib.YT_F64):
        self.lib = _lib.load()
        self.names = [t[0] for t in tensors]
        self.shapes = [tuple(int(x) for x in t[1]) for t in tensors]
        self.per_element = [t[3] is None for t in tensors]
        self._keep = []
        descs = (_lib.TensorDesc * len(tensors))()
        for i, (name, shape, pattern, values) in enumerate(tensors):
            shp = np.ascontiguousarray(shape, dtype=np.int32)
            self._keep.append(shp)
            d = descs[i]
            d.name = name.encode()
            d.ndim = len(shape)
            d.shape = shp.ctypes.data_as(C.POINTER(C.c_int32))
            if pattern is not None:
                pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.uint8).reshape(shape).ravel(order="F"))
                self._keep.append(pat)
                d.pattern = pat.ctypes.data_as(C.POINTER(C.c_uint8))
            if values is not None:
                val = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(shape).ravel(order="F"))
                self._keep.append(val)
                d.values = val.ctypes.data_as(C.POINTER(C.c_double))
        handle = C.c_void_p()
        _lib.check(self.lib.yt_plan_create(expr.encode(), descs, len(tensors), precision,
                                           C.byref(handle)), "yt_plan_create")
        self.handle = handle
        self.precision = precision

    def close(self):
        if getattr(self, "handle", None):
            self.lib.yt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = _lib.PlanStats()
        _lib.check(self.lib.yt_plan_stats_get(self.handle, C.byref(s)), "yt_plan_stats_get")
        return dict(nz_flops=s.nz_flops, hw_flops=s.hw_flops, naive_flops=s.naive_flops,
                    bytes_per_element=s.bytes_per_element, n_ops=s.n_ops, n_terms=s.n_terms,
                    log_cost=tuple(s.log_cost),
                    order=s.order.decode())

    def eqspp(self, term: int, name: str) -> np.ndarray:
        i = self.names.index(name)
        shape = self.shapes[i]
        out = np.zeros(int(np.prod(shape)), dtype=np.uint8)
        _lib.check(self.lib.yt_plan_eqspp(self.handle, term, i, out.ctypes.data_as(C.POINTER(C.c_uint8))),
                   "yt_plan_eqspp")
        return out.reshape(shape, order="F").astype(bool)

    def execute_ptrs(self, ptrs, n_elements: int, stream=None):
        """ptrs: one device pointer (int) per descriptor (ignored for constants)."""
        arr = (C.c_void_p * len(ptrs))(*[C.c_void_p(p) if p else None for p in ptrs])
        _lib.check(self.lib.yt_execute_batched(self.handle, arr, int(n_elements), _stream_handle(stream)),
                   "yt_execute_batched")

    def execute(self, tensors: dict, n_elements: int, stream=None):
        """tensors: name -> torch tensor on the GPU holding n_elements element tensors,
        each stored column-major (use element_major() to build them)."""
        ptrs = [tensors[n].data_ptr() if pe else 0 for n, pe in zip(self.names, self.per_element)]
        self.execute_ptrs(ptrs, n_elements, stream)


def element_major(arr: np.ndarray) -> np.ndarray:
    """(E, *shape) C-ordered numpy array -> flat buffer of E column-major element tensors."""
    E = arr.shape[0]
    return np.ascontiguousarray(arr.reshape(E, -1, order="C").reshape((E,) + arr.shape[1:])
                                .transpose([0] + list(range(arr.ndim - 1, 0, -1)))).reshape(E, -1)


def from_element_major(buf: np.ndarray, shape) -> np.ndarray:
    E = buf.shape[0]
    rev = tuple(reversed(shape))
    return np.ascontiguousarray(buf.reshape((E,) + rev).transpose([0] + list(range(len(shape), 0, -1))))
