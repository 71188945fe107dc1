"""Builds libpmc.so (the engine's C ABI, include/pmc.h) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel, then linked into one shared
library next to this file.  `python -m paper_1409_8336_gb300.build` rebuilds.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpmc.so")
# The engine is built twice: with IEEE single-precision math, and with
# -use_fast_math (hardware approximations of division, sqrt, log, exp, sin/cos),
# the build option the method's authors timed and verified equivalent.
VARIANTS = {"libpmc.so": [], "libpmc_fast.so": ["-use_fast_math"]}
SOURCES = ["transport.cu", "drain.cu", "cascade.cu", "stats.cu", "surrogate.cu", "gamma.cu", "host.cu"]
HEADERS = ["pmc_device.cuh", "pmc_kernels.cuh", "transport_step.cuh", "cascade_event.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def flags(extra=()):
    # host FP64 (physics tables, gamma offsets) must not be contracted into FMAs: the
    # aarch64 and x86-64 builds then give identical tables
    return [*ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I",
            os.path.join(ROOT, "include"), *extra]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "pmc.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, extra=(), out_dir: str | None = None):
    """Compiles every variant; returns the path of the default library."""
    out_dir = out_dir or HERE
    jobs, links = [], []
    for lib_name, vflags in VARIANTS.items():
        bdir = os.path.join(BUILD if out_dir == HERE else os.path.join(out_dir, "_build"), lib_name.split(".")[0])
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for s in SOURCES:
            src = os.path.join(CSRC, s)
            obj = os.path.join(bdir, s.replace(".cu", ".o"))
            objs.append(obj)
            if force or ptxas_info or extra or _stale(obj, src):
                px = ["-Xptxas", "-v"] if ptxas_info else []
                jobs.append((obj, [nvcc(), *flags([*vflags, *px, *extra]), "-c", src, "-o", obj]))
        links.append((os.path.join(out_dir, lib_name), objs))

    def run(job):
        obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (obj, r.stdout, r.stderr))
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out:
                print(out)
    for lib, objs in links:
        if jobs or not os.path.exists(lib):
            tmp = lib + ".tmp%d" % os.getpid()
            subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
            os.replace(tmp, lib)
    return os.path.join(out_dir, "libpmc.so")


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
