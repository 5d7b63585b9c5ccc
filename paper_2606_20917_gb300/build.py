"""Build libnir.so in-tree for sm_103a (nvcc, one process per translation unit).

The elemental-operator kernels are instantiated by ``csrc/nir_inst.cu`` and the
threading-over-elements Helmholtz kernels by ``csrc/nir_toe.cu``, each compiled
once per (shape, precision) so the units compile in parallel.
Usage: ``python paper_2606_20917_gb300/build.py [--force] [--jobs N]``.
"""
from __future__ import annotations

import argparse
import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnir.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", CSRC,
                  "-I", os.path.join(os.path.dirname(HERE), "include")]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libnir.so")


def _units():
    units = []
    for s in range(6):   # quad, tri, hex, prism, tet, pyramid
        for p in range(3):
            units.append((os.path.join(CSRC, "nir_inst.cu"), f"inst_s{s}_p{p}.o",
                          [f"-DNIR_SHAPE={s}", f"-DNIR_PREC={p}"]))
    for s in range(5):   # no threading-over-elements kernel for pyramids
        for p in range(3):
            units.append((os.path.join(CSRC, "nir_toe.cu"), f"toe_s{s}_p{p}.o",
                          [f"-DNIR_SHAPE={s}", f"-DNIR_PREC={p}"]))
    for d in (2, 3):
        for p in range(3):
            units.append((os.path.join(CSRC, "nir_mesh_inst.cu"), f"mesh_d{d}_p{p}.o",
                          [f"-DNIR_MESH_DIM={d}", f"-DNIR_PREC={p}"]))
    for src in ("nir_api.cu", "nir_geom.cu", "nir_solve.cu", "nir_cg.cu", "nir_asm.cu", "nir_noalloc.cu",
                "nir_basis.cpp", "nir_partition.cpp"):
        units.append((os.path.join(CSRC, src), os.path.splitext(src)[0] + ".o", []))
    return units


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h"))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    todo = []
    objs = []
    for src, obj, extra in _units():
        out = os.path.join(OBJ, obj)
        objs.append(out)
        if force or _stale(out, src):
            lang = ["-x", "cu"] if src.endswith(".cu") else []
            todo.append([nvcc] + NVFLAGS + extra + lang + ["-c", src, "-o", out])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)
        return cmd[-1]

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
            list(ex.map(run, todo))
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("-v", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, jobs=a.jobs, verbose=a.v))
