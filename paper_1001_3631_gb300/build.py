"""Compile the CUDA sources under csrc/ into the in-tree shared libraries libteuk.so and
libteuk_check.so (the same sources with TEUK_CHECK defined: device-side index checks
that report through the status word, see include/teuk.h).

nvcc -gencode arch=compute_103a,code=sm_103a (GB300) only; the translation units of both
libraries are compiled in parallel, then each is linked with a static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libteuk.so")
VARIANTS = {   # name: (library, object folder, extra flags)
    "release": (LIB, BUILD, []),
    "check": (os.path.join(HERE, "libteuk_check.so"), os.path.join(HERE, "_build_check"), ["-DTEUK_CHECK"]),
}
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "teuk.h")]


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), variants=("release", "check")) -> str:
    """Build the named variants that are out of date; returns the release library's path."""
    todo = [v for v in variants if force or _stale(VARIANTS[v][0])]
    if not todo:
        return LIB
    srcs = _sources()
    jobs = []
    for v in todo:
        lib, folder, flags = VARIANTS[v]
        os.makedirs(folder, exist_ok=True)
        for src in srcs:
            jobs.append((src, os.path.join(folder, os.path.basename(src)[:-3] + ".o"), flags))

    def compile_one(job):
        src, obj, flags = job
        cmd = [NVCC, *ARCH, *FLAGS, *flags, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return r.stdout + r.stderr

    # the largest translation units first, so that they do not finish last
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with cf.ThreadPoolExecutor(max_workers=min(max(os.cpu_count() or 8, 8), len(jobs))) as ex:
        logs = list(ex.map(compile_one, jobs))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    for v in todo:
        lib, folder, _ = VARIANTS[v]
        objs = [os.path.join(folder, os.path.basename(src)[:-3] + ".o") for src in srcs]
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra=sys.argv[1:]))
