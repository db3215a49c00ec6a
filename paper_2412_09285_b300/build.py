"""Build libfem.so in-tree with nvcc for sm_103a (B300).

``python -m paper_2412_09285_b300.build`` compiles every ``csrc/*.cu`` to an object
under ``_build/`` (in parallel, only when stale) and links the shared library
next to this file.  The CUDA runtime is linked statically, so the library needs
only the NVIDIA driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Code generation (single-precision denormals are kept: the step kernels flush them only
# in their approximate instructions, written with the .ftz forms in step_common.cuh).
CODEGEN = ["-O3", "-std=c++17", "-lineinfo"]
FLAGS = CODEGEN + ["-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "--expt-relaxed-constexpr",
                   "-I", INCLUDE, "-I", CSRC]
STAMP = os.path.join(BUILD, "flags.txt")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs


def _stale(obj, src, headers, flags_changed=False):
    if flags_changed or not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(x) > t for x in [src] + headers)


def build(verbose: bool = False, extra_flags=None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    headers = _headers()
    flags = FLAGS + list(extra_flags or [])
    # objects compiled with other code-generation flags are rebuilt
    stamp = " ".join(ARCH + CODEGEN + list(extra_flags or []))
    try:
        with open(STAMP) as fh:
            flags_changed = fh.read().strip() != stamp
    except OSError:
        flags_changed = True
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if _stale(o, s, headers, flags_changed):
            jobs.append([nvcc] + ARCH + flags + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return cmd[-3]

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        for done in ex.map(run, jobs):
            if verbose:
                print("compiled", os.path.basename(done), file=sys.stderr)
    if flags_changed:
        with open(STAMP, "w") as fh:
            fh.write(stamp + "\n")
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
