"""Build libtlfe.so (CUDA, sm_103a) in-tree.

Each translation unit under csrc/ is compiled by its own nvcc process (in
parallel), then linked into ``_build/libtlfe.so``. Re-running only recompiles
units whose source or any header is newer than their object file.

``build(checked=True)`` also links ``_build/libtlfe_checked.so``, the
bounds-checked build: the element-kernel units compiled with
TLFE_BOUNDS_CHECK (every index read from a device table range-checked into
the status word, see tlfe_internal.h), the other units shared with the
normal build. ``tlfe.load()`` takes it when TLFE_LIB names it.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtlfe.so")
LIB_CHECKED = os.path.join(OUT, "libtlfe_checked.so")
# units holding the element kernels: compiled a second time with the bounds checks
CHECKED_UNITS = ("k_force.cu", "k_matvec.cu", "k_vjp.cu", "k_diag.cu", "k_fm.cu", "k_fused_force.cu",
                 "k_fused_matvec.cu")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtlfe")


def _deps_mtime() -> float:
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hdrs.append(os.path.join(INCLUDE, "tlfe.h"))
    return max(os.path.getmtime(h) for h in hdrs)


def _compile(src: str, verbose_ptxas: bool, checked: bool = False) -> str:
    obj = os.path.join(OUT, os.path.basename(src).replace(".cu", ".checked.o" if checked else ".o"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _deps_mtime()):
        return obj
    extra = ["-DTLFE_BOUNDS_CHECK"] if checked else []
    cmd = [nvcc()] + ARCH + FLAGS + extra + (["-Xptxas", "-v"] if verbose_ptxas else []) + \
        ["-c", src, "-o", obj + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr[-4000:]}")
    if verbose_ptxas:
        with open(obj + ".ptxas.txt", "w") as fh:
            fh.write(res.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def _link(lib: str, objs) -> None:
    if os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(o) for o in objs):
        return
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + list(objs) + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
    os.replace(tmp, lib)


def build(verbose_ptxas: bool = False, jobs: int | None = None, checked: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    tasks = [(s, False) for s in srcs]
    if checked:
        tasks += [(s, True) for s in srcs if os.path.basename(s) in CHECKED_UNITS]
    # the heaviest units first, so that the parallel build ends sooner
    tasks.sort(key=lambda t: os.path.basename(t[0]) not in CHECKED_UNITS)
    jobs = jobs or min(len(tasks), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = dict(zip(tasks, ex.map(lambda t: _compile(t[0], verbose_ptxas, t[1]), tasks)))
    _link(LIB, [objs[(s, False)] for s in srcs])
    if checked:
        _link(LIB_CHECKED, [objs[(s, os.path.basename(s) in CHECKED_UNITS)] for s in srcs])
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, checked="--checked" in sys.argv))
