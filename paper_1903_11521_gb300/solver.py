"""Python view of the ADER-DG solver of the C ABI (argument marshalling only)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _stream_handle(stream) -> int | None:
    """A CUDA stream handle from a torch.cuda.Stream, an int, or None (default stream)."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Solver:
    """One elastic ADER-DG problem resident on the device.

    material (E,3) rho/lambda/mu; jacobian (E,3,3) dx/dxi; neighbours/faces/orient (E,4)
    or None.  DOFs are exchanged in the canonical layout [element][quantity][basis]."""

    def __init__(self, order, dt, material, jacobian, neighbours=None, faces=None,
                 orient=None, precision=_lib.YT_F64, stream=None, flags=0, attenuation=None, n_halo=0):
        """attenuation: None (elastic, 9 quantities) or an object with (E, 3) arrays
        omega, ylam, ymu of the three mechanisms (27 quantities)."""
        self.lib = _lib.load()
        E = int(np.asarray(material).shape[0])
        self.n_elements = E
        self.order = int(order)
        self._mat = np.ascontiguousarray(material, dtype=np.float64).reshape(E, 3)
        # column-major 3x3 per element: entry (i, c) at i + 3c
        self._jac = np.ascontiguousarray(np.asarray(jacobian, dtype=np.float64).reshape(E, 3, 3)
                                         .transpose(0, 2, 1)).reshape(E, 9)
        desc = _lib.MeshDesc()
        desc.n_elements = E
        desc.material = _ptr(self._mat, C.c_double)
        desc.jacobian = _ptr(self._jac, C.c_double)
        if neighbours is not None:
            self._nb = np.ascontiguousarray(neighbours, dtype=np.int32)
            self._fj = np.ascontiguousarray(faces, dtype=np.int8)
            self._fh = np.ascontiguousarray(orient, dtype=np.int8)
            desc.neighbours = _ptr(self._nb, C.c_int32)
            desc.faces = _ptr(self._fj, C.c_int8)
            desc.orient = _ptr(self._fh, C.c_int8)
        desc.n_halo = int(n_halo)
        self.n_quantities = 9
        if attenuation is not None:
            self._att = np.ascontiguousarray(np.stack([attenuation.omega, attenuation.ylam,
                                                       attenuation.ymu], axis=2), dtype=np.float64)
            assert self._att.shape == (E, 3, 3)
            desc.attenuation = _ptr(self._att, C.c_double)
            self.n_quantities = 27
        sch = _lib.SchemeDesc(order=self.order, dt=float(dt), precision=precision, flags=int(flags),
                              quantities=self.n_quantities)
        handle = C.c_void_p()
        _lib.check(self.lib.yt_solver_create(C.byref(desc), C.byref(sch),
                                             _stream_handle(stream), C.byref(handle)),
                   "yt_solver_create")
        self.handle = handle
        self.n_basis = (self.order) * (self.order + 1) * (self.order + 2) // 6

    def close(self):
        if getattr(self, "handle", None):
            self.lib.yt_solver_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ data movement
    def set_dofs_host(self, Q, stream=None):
        """Q as numpy (E, B, P) [element, basis, quantity] (the oracle's layout)."""
        canon = np.ascontiguousarray(np.asarray(Q, dtype=np.float64).transpose(0, 2, 1))
        self._host_in = canon
        _lib.check(self.lib.yt_solver_set_dofs(self.handle, canon.ctypes.data, _lib.YT_MEM_HOST,
                                               _stream_handle(stream)), "yt_solver_set_dofs")

    def set_dofs_ptr(self, ptr: int, where: int, stream=None):
        _lib.check(self.lib.yt_solver_set_dofs(self.handle, ptr, where, _stream_handle(stream)),
                   "yt_solver_set_dofs")

    def get_ptr(self, field: int, ptr: int, where: int, stream=None):
        _lib.check(self.lib.yt_solver_get(self.handle, field, ptr, where, _stream_handle(stream)),
                   "yt_solver_get")

    def get_host(self, field=_lib.YT_FIELD_DOFS, stream=None, sync=True):
        """Field as numpy (E, B, P); synchronises the device when sync is True."""
        out = np.empty((self.n_elements, self.n_quantities, self.n_basis))
        _lib.check(self.lib.yt_solver_get(self.handle, field, out.ctypes.data, _lib.YT_MEM_HOST,
                                          _stream_handle(stream)), "yt_solver_get")
        if sync:
            import torch
            torch.cuda.synchronize()
        return out.transpose(0, 2, 1)

    # ------------------------------------------------------------------------ compute
    def step(self, stream=None):
        _lib.check(self.lib.yt_step(self.handle, _stream_handle(stream)), "yt_step")

    def step_local(self, stream=None):
        _lib.check(self.lib.yt_step_local(self.handle, _stream_handle(stream)), "yt_step_local")

    def step_neighbour(self, stream=None):
        _lib.check(self.lib.yt_step_neighbour(self.handle, _stream_handle(stream)),
                   "yt_step_neighbour")

    def step_host_ptr(self, in_ptr: int, out_ptr: int, stream=None):
        """One step on host buffers (canonical layout), copies pipelined with the kernels."""
        _lib.check(self.lib.yt_step_host(self.handle, in_ptr, out_ptr, _stream_handle(stream)),
                   "yt_step_host")

    def step_phase(self, phase: int, stream=None):
        _lib.check(self.lib.yt_step_phase(self.handle, phase, _stream_handle(stream)), "yt_step_phase")

    def step_phase_tiles(self, phase: int, tile0: int, n_tiles: int, stream=None):
        _lib.check(self.lib.yt_step_phase_tiles(self.handle, phase, int(tile0), int(n_tiles),
                                                _stream_handle(stream)), "yt_step_phase_tiles")

    def set_send_list(self, pairs):
        """pairs: (n, 2) int (local element, face j) whose projections other ranks need."""
        self._send = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        _lib.check(self.lib.yt_solver_set_send_list(self.handle, _ptr(self._send, C.c_int32),
                                                    self._send.shape[0]), "yt_solver_set_send_list")

    def halo_pack(self, out_ptr: int, stream=None):
        _lib.check(self.lib.yt_solver_halo_pack(self.handle, out_ptr, _stream_handle(stream)),
                   "yt_solver_halo_pack")

    def halo_unpack(self, in_ptr: int, stream=None):
        _lib.check(self.lib.yt_solver_halo_unpack(self.handle, in_ptr, _stream_handle(stream)),
                   "yt_solver_halo_unpack")

    def status(self, stream=None):
        """Synchronises the stream; raises YtError (YT_ERR_TIMEOUT) if a bounded
        device-side wait of the tensor-core kernels ran out."""
        _lib.check(self.lib.yt_solver_status(self.handle, _stream_handle(stream)), "yt_solver_status")

    def stats(self):
        v = [C.c_double() for _ in range(4)]
        _lib.check(self.lib.yt_solver_stats(self.handle, *[C.byref(x) for x in v]),
                   "yt_solver_stats")
        return dict(local_flops=v[0].value, neighbour_flops=v[1].value,
                    local_bytes=v[2].value, neighbour_bytes=v[3].value)


def reference_matrix(order: int, name: str) -> np.ndarray:
    """Host-side reference matrix of the library (no device work)."""
    lib = _lib.load()
    n = C.c_int64()
    _lib.check(lib.yt_reference_matrix(order, name.encode(), None, C.byref(n)), "yt_reference_matrix")
    out = np.empty(n.value)
    _lib.check(lib.yt_reference_matrix(order, name.encode(), _ptr(out, C.c_double), C.byref(n)),
               "yt_reference_matrix")
    return out


class Batch:
    """p-adaptive mesh: per-element orders, one CUDA-graph launch per step.

    DOFs are exchanged as a list of (B_e, 9) arrays (the oracle's layout)."""

    def __init__(self, orders, dt, material, jacobian, neighbours, faces, orient,
                 precision=_lib.YT_F64, stream=None):
        self.lib = _lib.load()
        E = int(np.asarray(material).shape[0])
        self.n_elements = E
        self.orders = np.ascontiguousarray(orders, dtype=np.int8)
        self.nb = (self.orders.astype(np.int64) * (self.orders + 1) * (self.orders + 2)) // 6
        self.offsets = np.concatenate([[0], np.cumsum(9 * self.nb)])
        self._mat = np.ascontiguousarray(material, dtype=np.float64).reshape(E, 3)
        self._jac = np.ascontiguousarray(np.asarray(jacobian, dtype=np.float64).reshape(E, 3, 3)
                                         .transpose(0, 2, 1)).reshape(E, 9)
        self._nbr = np.ascontiguousarray(neighbours, dtype=np.int32)
        self._fj = np.ascontiguousarray(faces, dtype=np.int8)
        self._fh = np.ascontiguousarray(orient, dtype=np.int8)
        desc = _lib.MeshDesc(n_elements=E, material=_ptr(self._mat, C.c_double),
                             jacobian=_ptr(self._jac, C.c_double),
                             neighbours=_ptr(self._nbr, C.c_int32), faces=_ptr(self._fj, C.c_int8),
                             orient=_ptr(self._fh, C.c_int8))
        sch = _lib.SchemeDesc(order=0, dt=float(dt), precision=precision, flags=0)
        handle = C.c_void_p()
        _lib.check(self.lib.yt_batch_create(C.byref(desc), _ptr(self.orders, C.c_int8), C.byref(sch),
                                            _stream_handle(stream), C.byref(handle)), "yt_batch_create")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            self.lib.yt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, Q_list) -> np.ndarray:
        return np.concatenate([np.asarray(q, dtype=np.float64).T.ravel() for q in Q_list])

    def unpack(self, flat):
        return [flat[self.offsets[e]:self.offsets[e + 1]].reshape(9, self.nb[e]).T
                for e in range(self.n_elements)]

    def set_dofs_host(self, Q_list, stream=None):
        self._host_in = np.ascontiguousarray(self.pack(Q_list))
        _lib.check(self.lib.yt_batch_set_dofs(self.handle, self._host_in.ctypes.data, _lib.YT_MEM_HOST,
                                              _stream_handle(stream)), "yt_batch_set_dofs")

    def set_dofs_ptr(self, ptr, where, stream=None):
        _lib.check(self.lib.yt_batch_set_dofs(self.handle, ptr, where, _stream_handle(stream)), "yt_batch_set_dofs")

    def get_ptr(self, field, ptr, where, stream=None):
        _lib.check(self.lib.yt_batch_get(self.handle, field, ptr, where, _stream_handle(stream)), "yt_batch_get")

    def get_host(self, field=_lib.YT_FIELD_DOFS, stream=None):
        out = np.empty(int(self.offsets[-1]))
        _lib.check(self.lib.yt_batch_get(self.handle, field, out.ctypes.data, _lib.YT_MEM_HOST,
                                         _stream_handle(stream)), "yt_batch_get")
        import torch
        torch.cuda.synchronize()
        return self.unpack(out)

    def step(self, stream=None):
        _lib.check(self.lib.yt_batch_step(self.handle, _stream_handle(stream)), "yt_batch_step")

    def tune(self, repeats=5, stream=None) -> int:
        chosen = C.c_int32()
        _lib.check(self.lib.yt_batch_tune(self.handle, repeats, _stream_handle(stream), C.byref(chosen)),
                   "yt_batch_tune")
        return chosen.value

    def set_form(self, form: int, order: int = 0, chunk: int = 1):
        """0: per-degree kernels in sequence, 1: on parallel branches, 2: the persistent
        kernel (order 0 by decreasing degree / 1 interleaved, chunk tiles per claim)."""
        _lib.check(self.lib.yt_batch_set_form(self.handle, form, order, chunk), "yt_batch_set_form")

    def config(self) -> str:
        buf = C.create_string_buffer(4096)
        _lib.check(self.lib.yt_batch_config(self.handle, buf, 4096), "yt_batch_config")
        return buf.value.decode()

    def status(self, stream=None):
        """Synchronises; raises YtError (YT_ERR_TIMEOUT) if the persistent kernel's grid
        barrier ran out."""
        _lib.check(self.lib.yt_batch_status(self.handle, _stream_handle(stream)), "yt_batch_status")

    def stats(self):
        f, b, g = C.c_double(), C.c_double(), C.c_int32()
        _lib.check(self.lib.yt_batch_stats(self.handle, C.byref(f), C.byref(b), C.byref(g)), "yt_batch_stats")
        return dict(flops=f.value, bytes=b.value, groups=g.value)


class Server:
    """Continuous-batching server of independent solves (see yt_server_* in the C ABI)."""

    def __init__(self, hbm_budget_bytes: int, precision=_lib.YT_F32):
        self.lib = _lib.load()
        desc = _lib.ServerDesc(hbm_budget_bytes=int(hbm_budget_bytes), precision=precision, flags=0)
        handle = C.c_void_p()
        _lib.check(self.lib.yt_server_create(C.byref(desc), C.byref(handle)), "yt_server_create")
        self.handle = handle
        self._shapes = {}

    def submit(self, order, dt, material, jacobian, neighbours, faces, orient, Q, steps) -> int:
        """Q: numpy (E, B, 9) [element, basis, quantity]; returns the request id."""
        E = int(np.asarray(material).shape[0])
        mat = np.ascontiguousarray(material, dtype=np.float64).reshape(E, 3)
        jac = np.ascontiguousarray(np.asarray(jacobian, dtype=np.float64).reshape(E, 3, 3)
                                   .transpose(0, 2, 1)).reshape(E, 9)
        nb = np.ascontiguousarray(neighbours, dtype=np.int32)
        fj = np.ascontiguousarray(faces, dtype=np.int8)
        fh = np.ascontiguousarray(orient, dtype=np.int8)
        canon = np.ascontiguousarray(np.asarray(Q, dtype=np.float64).transpose(0, 2, 1))
        desc = _lib.MeshDesc(n_elements=E, material=_ptr(mat, C.c_double), jacobian=_ptr(jac, C.c_double),
                             neighbours=_ptr(nb, C.c_int32), faces=_ptr(fj, C.c_int8),
                             orient=_ptr(fh, C.c_int8))
        rid = C.c_int64()
        _lib.check(self.lib.yt_server_submit(self.handle, C.byref(desc), int(order), float(dt),
                                             canon.ctypes.data, int(steps), C.byref(rid)),
                   "yt_server_submit")
        self._shapes[rid.value] = (E, canon.shape[2])
        return rid.value

    def wait(self, rid: int):
        """(Q (E, B, 9), latency s, queue s)."""
        E, B = self._shapes[rid]
        out = np.empty((E, 9, B))
        lat, q = C.c_double(), C.c_double()
        _lib.check(self.lib.yt_server_wait(self.handle, rid, out.ctypes.data, C.byref(lat), C.byref(q)),
                   "yt_server_wait")
        return out.transpose(0, 2, 1), lat.value, q.value

    def fail_tick(self, at_tick: int):
        """Diagnostics: the worker treats its step `at_tick` as failed (host side)."""
        _lib.check(self.lib.yt_server_fail_tick(self.handle, int(at_tick)), "yt_server_fail_tick")

    def stats(self) -> dict:
        st = _lib.ServerStats()
        _lib.check(self.lib.yt_server_stats_get(self.handle, C.byref(st)), "yt_server_stats_get")
        return {n: getattr(st, n) for n, _ in _lib.ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.yt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
