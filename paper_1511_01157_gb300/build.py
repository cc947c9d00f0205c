"""Build libmorse.so in-tree with nvcc for sm_103a (GB300).

Each .cu translation unit compiles in parallel to an object, then one link
step makes the shared library next to this file.  No cmake, one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libmorse.so")
OUT_CHECKED = os.path.join(HERE, "libmorse_checked.so")
BUILD = os.path.join(HERE, "_build", platform.machine())  # per host arch
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith(".cu"))


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _build_one(out, objdir, force, verbose, extra):
    os.makedirs(objdir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
               if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "morse.h"))
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", INCLUDE, "-I", CSRC] + list(extra)
    if verbose:
        flags += ["-Xptxas", "-v"]
    objs, jobs = [], []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc(), "-c", src, "-o", obj] + flags)
    return objs, jobs, out


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" +
                           r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, extra=(),
          checked: bool = True) -> str:
    """Build libmorse.so and, unless checked=False, libmorse_checked.so
    (every texel index checked in device code; for tests)."""
    variants = [_build_one(OUT, BUILD, force, verbose, extra)]
    if checked:
        variants.append(_build_one(OUT_CHECKED, BUILD + "_checked", force,
                                   False, list(extra) +
                                   ["-DMORSE_CHECK_BOUNDS"]))
    jobs = [j for v in variants for j in v[1]]
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose:
        for line in logs:
            sys.stdout.write(line)
    for objs, vjobs, out in variants:
        if force or vjobs or _stale(out, objs):
            tmp = out + ".tmp"
            _run([nvcc(), "-shared"] + ARCH + objs +
                 ["-o", tmp, "-cudart", "static"])
            os.replace(tmp, out)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
