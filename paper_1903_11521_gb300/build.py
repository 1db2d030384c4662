"""Builds the in-tree shared library ``_build/libyateto_gb300.so`` with nvcc for sm_103a.

Every translation unit under ``csrc/`` is compiled in parallel, then linked into one
shared library against the shared CUDA runtime.  Nothing is installed.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libyateto_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + CSRC, "-I" + os.path.join(BUILD, "gen")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build yateto_gb300")
    return path


def sources():
    sys.path.insert(0, HERE)
    import codegen
    generated = codegen.generate(BUILD)
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp"))) + generated


# Units named *_rdc.cu (the persistent batch kernel and its per-degree tile functions) are
# compiled for separate compilation and device-linked together; every other unit is a
# whole-program unit.  Their functions are capped at 168 registers: the kernel calling
# them runs 288 threads (9 warps) per CTA, 3 warps on one SM sub-partition.
RDC_FLAGS = ["-rdc=true", "-maxrregcount=168"]


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    if src.endswith("_rdc.cu"):
        extra = RDC_FLAGS + extra
    gen = os.path.join(BUILD, "gen")
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    if os.path.isdir(gen):
        deps += [os.path.join(gen, h) for h in os.listdir(gen) if h.endswith(".cuh")]
    deps.append(os.path.join(HERE, "..", "include", "yateto_gb300.h"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-x", "cu", *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    extra = extra or []
    # the largest units (highest degree) first, so that they do not finish last
    def cost(src):
        m = re.search(r"ader_o(\d)_", os.path.basename(src))
        return -(int(m.group(1)) if m else 0)
    srcs = sorted(sources(), key=cost)
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    rdc = [o for o in objs if o.endswith("_rdc.cu.o")]
    dlink = os.path.join(BUILD, "batch_dlink.o")
    if rdc and (not os.path.exists(dlink) or os.path.getmtime(dlink) < max(os.path.getmtime(o) for o in rdc)):
        res = subprocess.run([nvcc(), *ARCH, "-Xcompiler", "-fPIC", "-dlink", *rdc, "-o", dlink],
                             capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"device link failed:\n{res.stdout}\n{res.stderr}")
    if rdc:
        objs = objs + [dlink]
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
