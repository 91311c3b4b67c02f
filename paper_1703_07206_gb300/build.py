"""Build libsgml.so (CUDA, sm_103a) in-tree with nvcc.

The kernel unit is compiled once per column-tile width (32 x 16 and 64 x 8 tiles, namespaces
``sgml_t32`` / ``sgml_t64``), the host units once; the objects are compiled in parallel and
linked into ``paper_1703_07206_gb300/_build/libsgml.so``.  Cross-compiles without a GPU.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libsgml.so")
# (source, object tag, extra defines): the cycle kernels are compiled once per tile width
UNITS = [
    ("sgml_kernels.cu", "k32", ["SGML_TILE_X=32", "SGML_KNS=sgml_t32"]),
    ("sgml_kernels.cu", "k64", ["SGML_TILE_X=64", "SGML_KNS=sgml_t64", "SGML_DEFINE_COMMON"]),
    ("sgml_api.cu", "api", []),
    ("sgml_noalloc.cu", "noalloc", []),
    ("sgml_post.cu", "post", []),
    ("sgml_peaks.cu", "peaks", []),
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "sgml.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, defines=(), out: str | None = None) -> str:
    """Compile libsgml.so if any source changed (or force).  Returns the library path.  `defines`
    (e.g. ["SGML_SWEEP_STAGES=8"]) and `out` build a variant elsewhere (tuning experiments)."""
    lib = out or LIB
    if not force and out is None and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, "-Xptxas", "-v"]
    flags += [f"-D{d}" for d in defines]

    def compile_one(unit):
        src, tag, defs = unit
        obj = os.path.join(BUILD, f"{tag}.{os.getpid()}.{abs(hash(lib))}.o")
        r = subprocess.run([cc, *flags, *[f"-D{d}" for d in defs], "-c", os.path.join(CSRC, src), "-o", obj],
                           capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise subprocess.CalledProcessError(r.returncode, r.args)
        if verbose:
            sys.stderr.write(r.stderr)
        if out is None:  # ptxas's resource report (registers, spills, shared memory) of the build
            with open(os.path.join(BUILD, f"ptxas_{tag}.log"), "w") as fh:
                fh.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
