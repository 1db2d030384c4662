"""Build-time generator of the unrolled sparse loops of the ADER-DG kernels.

For every polynomial degree N = 1..6 it emits ``_build/gen/yt_rows_o{N}.cuh`` with one
specialisation ``Row<N, LIST, ROW>`` per row of every sparse list of the step (the CK
derivative lists Ktilde^x restricted to the staircase, Khat^x, R^sT and Rhat^s): a
straight-line sum over the row's non-zeros, values read at fixed offsets of the value
array the solver uploads and operands at fixed offsets of the per-thread shared-memory
column.  The sparsity patterns come from the library's own reference matrices (through a
host-only helper library), and the value offsets follow the order in which the solver
packs its CSR lists: derivative lists (delta, x), volume lists (x), then for every face
R^sT and Rhat^s; rows in order, columns ascending.  ``ader_o{N}_{prec}_{variant}.cu`` instantiates
one kernel variant of that degree and precision in its own translation unit, so that the
units compile in parallel.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ORDERS_N = (1, 2, 3, 4, 5, 6)
# (degree, contraction type) pairs that get kernels
UNITS = [(n, "f64") for n in (1, 2, 3, 4, 5, 6)] + [(n, "f32") for n in (1, 2, 3, 4, 5, 6)]
ROW_STRIDE = 9 * 32          # doubles between consecutive rows of a thread's column
N_ACC = 4


def host_helper(build_dir: str) -> str:
    out = os.path.join(build_dir, "libyt_tables_host.so")
    srcs = [os.path.join(CSRC, "tables.cpp"), os.path.join(CSRC, "host_tools", "tables_export.cpp")]
    if not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(s) for s in
                                                               srcs + [os.path.join(CSRC, "tables.h")]):
        cxx = os.environ.get("CXX", "g++")
        res = subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", *srcs, "-o", out],
                             capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"host helper build failed:\n{res.stderr}")
    return out


def matrices(lib, N):
    B = (N + 1) * (N + 2) * (N + 3) // 6
    BT = (N + 1) * (N + 2) // 2

    def get(name, count, shape):
        buf = np.empty(count)
        n = C.c_int64()
        rc = lib.yt_host_reference_matrix(N, name.encode(), buf.ctypes.data_as(C.POINTER(C.c_double)),
                                          C.byref(n))
        if rc != 0 or n.value != count:
            raise RuntimeError(f"reference matrix {name} of degree {N}: status {rc}")
        return buf.reshape(shape)        # stacked, each column-major: [.., col, row]

    Kt = get("Ktilde", 3 * B * B, (3, B, B))
    Kh = get("Khat", 3 * B * B, (3, B, B))
    R = get("R", 4 * BT * B, (4, BT, B))
    Rh = get("Rhat", 4 * BT * B, (4, BT, B))
    return B, BT, Kt, Kh, R, Rh


def lists(N, B, BT, Kt, Kh, R, Rh):
    """[(list_id, rows)] in packing order; rows[r] = [(col, value_offset)]."""
    nd = lambda d: (N - d + 3) * (N - d + 2) * (N - d + 1) // 6
    out = []
    off = 0

    def add(list_id, nrows, ncols, at):
        nonlocal off
        rows = []
        for r in range(nrows):
            row = []
            for c in range(ncols):
                if at(r, c) != 0.0:
                    row.append((c, off))
                    off += 1
            rows.append(row)
        out.append((list_id, rows))

    for d in range(N):
        for x in range(3):
            add(d * 3 + x, nd(d + 1), nd(d), lambda r, c, x=x: Kt[x][c, r])
    for x in range(3):
        add(18 + x, B, B, lambda r, c, x=x: Kh[x][c, r])
    for f in range(4):
        add(21 + f, BT, B, lambda r, c, f=f: R[f][r, c])       # R^sT: row m, column l
        add(25 + f, B, BT, lambda r, c, f=f: Rh[f][c, r])      # Rhat^s: row k, column m
    return out, off


CONST_MAX_N = 5          # FP32 values of degrees <= 5 fit the 64 KB constant bank


def emit_rows(N, lst, nvals):
    lines = []
    if N <= CONST_MAX_N:
        # FP32 values in constant memory: each non-zero becomes one fma with a
        # constant-bank operand (one copy per translation unit, uploaded by the solver);
        # not in the batch kernel's units (YT_ROWS_GLOBAL)
        lines.append("#ifndef YT_ROWS_GLOBAL")
        lines.append(f"static __constant__ float c_vals_o{N}[{max(nvals, 1)}];")
        lines.append("#endif")
    for list_id, rows in lst:
        for r, row in enumerate(rows):
            lines.append(f"template <> struct Row<{N}, {list_id}, {r}> {{")
            lines.append("  template <typename R>")
            lines.append("  static __device__ __forceinline__ R dot(const R* __restrict__ v, "
                         "const R* __restrict__ x) {")
            if not row:
                lines.append("    return R(0);")
            else:
                na = min(N_ACC, len(row))
                for a in range(na):
                    lines.append(f"    R a{a} = R(0);")
                for i, (c, voff) in enumerate(row):
                    a = i % na
                    lines.append(f"    a{a} = fma(__ldg(v + {voff}), x[{c * ROW_STRIDE}], a{a});")
                terms = [f"a{a}" for a in range(na)]
                while len(terms) > 1:
                    terms = [f"({terms[i]} + {terms[i + 1]})" if i + 1 < len(terms) else terms[i]
                             for i in range(0, len(terms), 2)]
                lines.append(f"    return {terms[0]};")
            lines.append("  }")
            # one accumulator continuing from `a` (FP64: the pipe, not latency, is the
            # limit, and every extra accumulator costs an add to combine)
            lines.append("  template <typename R>")
            lines.append("  static __device__ __forceinline__ R dot1(const R* __restrict__ v, "
                         "const R* __restrict__ x, R a) {")
            for c, voff in row:
                lines.append(f"    a = fma(__ldg(v + {voff}), x[{c * ROW_STRIDE}], a);")
            lines.append("    return a;")
            lines.append("  }")
            # the same two forms with the operand column in a register array x[0..S)
            lines.append("  template <typename R, int S>")
            lines.append("  static __device__ __forceinline__ R dotr1(const R* __restrict__ v, "
                         "const R (&x)[S], R a) {")
            for c, voff in row:
                lines.append(f"    a = fma(__ldg(v + {voff}), x[{c}], a);")
            lines.append("    return a;")
            lines.append("  }")
            # operand rows c < S in the register array, rows c >= S in shared memory
            lines.append("  template <typename R, int S>")
            lines.append("  static __device__ __forceinline__ R dotrh(const R* __restrict__ v, "
                         "const R (&xr)[S], const R* __restrict__ xs, R a) {")
            for c, voff in row:
                lines.append(f"    a = fma(__ldg(v + {voff}), ({c} < S) ? xr[({c} < S) ? {c} : 0] : "
                             f"xs[({c} - S) * {ROW_STRIDE}], a);")
            lines.append("    return a;")
            lines.append("  }")
            if N <= CONST_MAX_N:
                lines.append("#ifndef YT_ROWS_GLOBAL")
                lines.append("  template <int S>")
                lines.append("  static __device__ __forceinline__ float dotrc(const float (&x)[S]) {")
                if not row:
                    lines.append("    return 0.0f;")
                else:
                    na = min(N_ACC, len(row))
                    for a in range(na):
                        lines.append(f"    float a{a} = 0.0f;")
                    for i, (c, voff) in enumerate(row):
                        a = i % na
                        lines.append(f"    a{a} = fmaf(c_vals_o{N}[{voff}], x[{c}], a{a});")
                    terms = [f"a{a}" for a in range(na)]
                    while len(terms) > 1:
                        terms = [f"({terms[i]} + {terms[i + 1]})" if i + 1 < len(terms) else terms[i]
                                 for i in range(0, len(terms), 2)]
                    lines.append(f"    return {terms[0]};")
                lines.append("  }")
            if N <= CONST_MAX_N:
                lines.append("  static __device__ __forceinline__ float dotc(const float* __restrict__ x) {")
                if not row:
                    lines.append("    return 0.0f;")
                else:
                    na = min(N_ACC, len(row))
                    for a in range(na):
                        lines.append(f"    float a{a} = 0.0f;")
                    for i, (c, voff) in enumerate(row):
                        a = i % na
                        lines.append(f"    a{a} = fmaf(c_vals_o{N}[{voff}], x[{c * ROW_STRIDE}], a{a});")
                    terms = [f"a{a}" for a in range(na)]
                    while len(terms) > 1:
                        terms = [f"({terms[i]} + {terms[i + 1]})" if i + 1 < len(terms) else terms[i]
                                 for i in range(0, len(terms), 2)]
                    lines.append(f"    return {terms[0]};")
                lines.append("  }")
                lines.append("#endif")
            lines.append("};")
    return "\n".join(lines) + "\n"


VARIANTS = {"lf": ("true", "true"), "ll": ("true", "false"), "nf": ("false", "true"),
            "np": ("false", "false")}
# kernels of a 27-quantity step: local (VE), neighbour flux of the elastic rows, anelastic rows
VE_VARIANTS = {"vl": 0, "vn": 1, "vt": 2}

UNIT = """// Generated by codegen.py: one kernel variant ({V}) of polynomial degree {N},
// contraction type {REAL}.
#include "ader_kernels.cuh"
#include "yt_rows_o{N}.cuh"

namespace yt {{
void ader_set_attribute_o{N}_{P}_{V}(size_t smem) {{ ader_set_attribute<{N}, {REAL}, {LOCAL}, {FUSED}>(smem); }}
void ader_launch_o{N}_{P}_{V}(const AderLaunch& L) {{ ader_launch<{N}, {REAL}, {LOCAL}, {FUSED}>(L); }}
int ader_upload_o{N}_{P}_{V}(const float* vals, size_t n) {{ {UPLOAD} }}
}}  // namespace yt
"""

VE_UNIT = """// Generated by codegen.py: one kernel of a 27-quantity step ({V}) of polynomial degree
// {N}, contraction type {REAL}.
#include "ader_kernels.cuh"
#include "yt_rows_o{N}.cuh"

namespace yt {{
void ader_set_attribute_o{N}_{P}_{V}(size_t smem) {{ ader_set_attribute_ve<{N}, {REAL}, {WHICH}>(smem); }}
void ader_launch_o{N}_{P}_{V}(const AderLaunch& L) {{ ader_launch_ve<{N}, {REAL}, {WHICH}>(L); }}
int ader_upload_o{N}_{P}_{V}(const float* vals, size_t n) {{ {UPLOAD} }}
}}  // namespace yt
"""

SMALL_UNIT = """// Generated by codegen.py: the small-mesh local update (k_local_small) of polynomial
// degree {N}, contraction type {REAL}.
#include "ader_kernels.cuh"
#include "yt_rows_o{N}.cuh"

namespace yt {{
void ader_set_attribute_o{N}_{P}_ls(size_t smem) {{ ader_set_attribute_small<{N}, {REAL}>(smem); }}
void ader_launch_o{N}_{P}_ls(const AderLaunch& L) {{ ader_launch_small<{N}, {REAL}>(L); }}
int ader_upload_o{N}_{P}_ls(const float* vals, size_t n) {{ {UPLOAD} }}
}}  // namespace yt
"""
# degrees with a small-mesh local kernel (the operand column fits the registers)
SMALL_MAX_N = 4

BATCH_UNIT = """// Generated by codegen.py: the tile functions of the persistent batch kernel for
// polynomial degree {N}, contraction type {REAL} (separately compiled, -rdc; values of the
// sparse rows from global memory).
#define YT_ROWS_GLOBAL 1
#include "batch_kernel.cuh"
#include "yt_rows_o{N}.cuh"

namespace yt {{
namespace {{
__device__ __forceinline__ StepTables<{REAL}> tables_of(const BatchGroup* g) {{
  StepTables<{REAL}> T;
  T.val = static_cast<const {REAL}*>(g->val);
  T.f = static_cast<const {REAL}*>(g->f);
  T.dt = g->dt;
  double f = 1.0;
  for (int i = 0; i < 8; ++i) {{
    f *= (i + 1.0);
    T.invfact[i] = 1.0 / f;
  }}
  return T;
}}
}}  // namespace

__device__ __noinline__ void batch_local_o{N}_{P}(const BatchGroup* g, const StarPattern* SP, size_t tile) {{
  local_tile<{N}, false, {REAL}, false>(g->Q, g->Q, g->I, static_cast<{REAL}*>(g->Pface),
                                        static_cast<{REAL}*>(g->Wloc), static_cast<const {REAL}*>(g->star),
                                        static_cast<const {REAL}*>(g->floc), tables_of(g), *SP,
                                        VeTables<{REAL}>{{}}, tile, g->dt);
}}

__device__ __noinline__ void batch_neigh_o{N}_{P}(const BatchGroup* g, const FaceGroups* G, size_t tile) {{
  neigh_tile<{N}, true, {REAL}, kNq>(g->Q, *G, static_cast<const {REAL}*>(g->Wloc),
                                     static_cast<const {REAL}*>(g->fnb), g->conn, tables_of(g), tile);
}}
}}  // namespace yt
"""

INFO = """// Generated by codegen.py: number of packed non-zero values per degree, checked by the
// solver against its own packing of the reference matrices.
namespace yt {{
int ader_generated_nnz(int N) {{
  switch (N) {{
{CASES}
  }}
  return -1;
}}
}}  // namespace yt
"""


def generate(build_dir: str) -> list[str]:
    gen = os.path.join(build_dir, "gen")
    os.makedirs(gen, exist_ok=True)
    lib = C.CDLL(host_helper(build_dir))
    lib.yt_host_reference_matrix.restype = C.c_int
    lib.yt_host_reference_matrix.argtypes = [C.c_int, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    units = []
    counts = {}
    for N in ORDERS_N:
        B, BT, Kt, Kh, R, Rh = matrices(lib, N)
        lst, nvals = lists(N, B, BT, Kt, Kh, R, Rh)
        counts[N] = nvals
        header = (f"// Generated by codegen.py: unrolled sparse rows of polynomial degree {N} "
                  f"({nvals} non-zeros).\n#pragma once\nnamespace yt {{\nnamespace gen {{\n"
                  + emit_rows(N, lst, nvals) + "}  // namespace gen\n}  // namespace yt\n")
        _write_if_changed(os.path.join(gen, f"yt_rows_o{N}.cuh"), header)
    for N, P in UNITS:
        for V, (local, fused) in VARIANTS.items():
            unit = os.path.join(gen, f"ader_o{N}_{P}_{V}.cu")
            if P == "f32" and N <= CONST_MAX_N:
                upload = (f"return (int)cudaMemcpyToSymbol(gen::c_vals_o{N}, vals, n * sizeof(float));")
            else:
                upload = "(void)vals; (void)n; return 0;"
            _write_if_changed(unit, UNIT.format(N=N, P=P, V=V, LOCAL=local, FUSED=fused, UPLOAD=upload,
                                                REAL="double" if P == "f64" else "float"))
            units.append(unit)
        if N <= SMALL_MAX_N:
            unit = os.path.join(gen, f"ader_o{N}_{P}_ls.cu")
            if P == "f32" and N <= CONST_MAX_N:
                upload = (f"return (int)cudaMemcpyToSymbol(gen::c_vals_o{N}, vals, n * sizeof(float));")
            else:
                upload = "(void)vals; (void)n; return 0;"
            _write_if_changed(unit, SMALL_UNIT.format(N=N, P=P, UPLOAD=upload,
                                                      REAL="double" if P == "f64" else "float"))
            units.append(unit)
        unit = os.path.join(gen, f"ader_o{N}_{P}_batch_rdc.cu")
        _write_if_changed(unit, BATCH_UNIT.format(N=N, P=P, REAL="double" if P == "f64" else "float"))
        units.append(unit)
        for V, which in VE_VARIANTS.items():
            unit = os.path.join(gen, f"ader_o{N}_{P}_{V}.cu")
            if P == "f32" and N <= CONST_MAX_N:
                upload = (f"return (int)cudaMemcpyToSymbol(gen::c_vals_o{N}, vals, n * sizeof(float));")
            else:
                upload = "(void)vals; (void)n; return 0;"
            _write_if_changed(unit, VE_UNIT.format(N=N, P=P, V=V, WHICH=which, UPLOAD=upload,
                                                   REAL="double" if P == "f64" else "float"))
            units.append(unit)
    info = os.path.join(gen, "ader_gen_info.cu")
    cases = "\n".join(f"    case {n}: return {c};" for n, c in counts.items())
    _write_if_changed(info, INFO.format(CASES=cases))
    units.append(info)
    return units


def _write_if_changed(path, text):
    if os.path.exists(path) and open(path).read() == text:
        return
    with open(path, "w") as f:
        f.write(text)
