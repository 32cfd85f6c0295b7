"""Builds ``libonng.so`` (the CUDA library behind ``include/onng.h``) in-tree.

Every translation unit in ``csrc/`` is compiled for sm_103a only, in parallel,
then linked into one shared library next to this file.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libonng.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(cuda, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


# Translation units compiled more than once, one object per flag set: the search
# kernels are instantiated per (vector type, chunks per lane, kept-list size) in
# separate objects so that they compile in parallel.
VARIANTS = {
    "search_inst.cu": [(f"t{t}_v{v}_k{kr}", [f"-DONNG_INST_T={t}", f"-DONNG_INST_V={v}", f"-DONNG_INST_KR={kr}"])
                       for t in (0, 1, 2) for v in (1, 2, 4, 8) for kr in (1, 4)],
}


LIB_CHECK = os.path.join(HERE, "libonng_check.so")
CHECK_FLAGS = ("-DONNG_CHECK",)


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _units(extra):
    """(source, object, flags) of every object the library links."""
    out = []
    checked = "-DONNG_CHECK" in extra
    for src in _sources():
        base = os.path.basename(src)[:-3]
        for tag, flags in VARIANTS.get(os.path.basename(src), [("", [])]):
            if checked and tag.startswith(("t1", "t2")):
                continue  # the bounds-checked build carries the float32 search only
            obj = os.path.join(BUILD, base + (f"_{tag}" if tag else "") + ".o")
            out.append((src, obj, flags + list(extra)))
    return out


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, lib: str = LIB, extra=()) -> str:
    """Compile the library if any source is newer than it; returns its path.

    ``lib`` / ``extra`` build a variant with extra nvcc flags (for instance a
    smaller tunable) under another name, in its own object folder."""
    if not force and not _stale(lib):
        return lib
    build_dir = BUILD if lib == LIB else os.path.join(BUILD, os.path.basename(lib).replace(".", "_"))
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(unit):
        src, obj, flags = unit
        obj = os.path.join(build_dir, os.path.basename(obj))
        cmd = [nvcc, *ARCH, *FLAGS, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {' '.join(flags)}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    units = _units(extra)
    # longest first: the search instantiations dominate
    units.sort(key=lambda u: os.path.basename(u[0]) != "search_inst.cu")
    with ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The bounds-checked library (-DONNG_CHECK): the search checks every id and
    row it reads from the graph and canary words between the warps' shared
    memory, flagging ONNG_FLAG_CHECK instead of reading out of bounds."""
    return build(force=force, verbose=verbose, lib=LIB_CHECK, extra=CHECK_FLAGS)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
