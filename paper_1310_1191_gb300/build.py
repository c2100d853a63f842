"""Build the in-tree CUDA library ``libfem_gb300.so`` for sm_103a with nvcc.

Each translation unit under ``csrc/`` is compiled in parallel into
``_build/`` and linked into a shared library next to this file.  The build is
incremental (an object is rebuilt when its source or any header is newer).

``build(checked=True)`` makes the checked variant ``libfem_gb300_checked.so``
(objects in ``_build_checked/``, compiled with ``-DFEM_CHECKED``): the same
entry points, with index checks in the kernels (element ids taken from
permutations, output offsets of mixed-degree plans) that skip a failing access
and report FEM_ECHECKED through ``fem_error_flag``.  ``_lib.load()`` picks it
when the environment sets ``FEM_GB300_CHECKED=1``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfem_gb300.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libfem_gb300_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build the library")
    return cand


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.inc")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max(os.path.getmtime(h) for h in hs) if hs else 0.0


def build(verbose: bool = False, jobs: int = 0, extra_flags=None, checked: bool = False) -> str:
    """Compile every source under csrc/ and link libfem_gb300.so (with
    ``checked``: libfem_gb300_checked.so); returns its path."""
    nvcc = _nvcc()
    bdir, lib_path = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr_t = _headers_mtime()
    flags = _flags() + (["-DFEM_CHECKED"] if checked else []) + list(extra_flags or [])

    def obj_of(s):
        return os.path.join(bdir, os.path.basename(s) + ".o")

    def compile_one(s):
        o = obj_of(s)
        if os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), hdr_t):
            return o, ""
        cmd = [nvcc] + flags + ["-c", s, "-o", o + ".tmp"]
        if s.endswith(".cpp"):
            cmd[1:1] = ["-x", "cu"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (s, r.stdout, r.stderr))
        os.replace(o + ".tmp", o)
        return o, r.stdout + r.stderr

    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for o, log in results:
            if log.strip():
                print(log)
    objs = [o for o, _ in results]
    if not os.path.exists(lib_path) or os.path.getmtime(lib_path) < max(os.path.getmtime(o) for o in objs):
        tmp = lib_path + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
            ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, checked="--checked" in sys.argv))
