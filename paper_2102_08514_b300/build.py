"""Build the CUDA library in-tree:  python -m paper_2102_08514_b300.build [--force] [--ptxas-v]

Compiles for sm_103a only.  The ABI (csrc/interp.cu) and one instantiation unit per (spline,
kernel family) (csrc/ops_inst.cu with -DINTERP_SPLINE / -DINTERP_PART) compile in parallel into
paper_2102_08514_b300/_build/obj/, then link into _build/libinterp_b300.so.  An object is rebuilt
when its command line or the contents of its sources changed (a stamp beside it).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
OUT = os.path.join(BUILD, "libinterp_b300.so")
GEN_HDR = os.path.join(CSRC, "generated", "splines.h")
COMMON_DEPS = [os.path.join(CSRC, f) for f in ("kernels.cuh", "registry.h", "layout.h", "ops_inst.cu", "batch_inst.cu", "interp.cu")] + \
    [GEN_HDR, os.path.join(ROOT, "include", "interp.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++20", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-O3"]
N_PARTS = 4


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def spline_names() -> list[str]:
    text = open(GEN_HDR).read()
    m = re.search(r"#define INTERP_GEN_SPLINES\(X\) (.*)", text)
    return re.findall(r"X\((\w+)\)", m.group(1))


STAMP = os.path.join(BUILD, "libinterp_b300.stamp")


def source_digest() -> str:
    """Hash of every source, header and flag the library depends on (file times need not survive
    a copy of the tree, contents do)."""
    h = hashlib.sha256(" ".join(NVCC_FLAGS).encode())
    for p in sorted(COMMON_DEPS):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_digest() -> str:
    """Hash of what the device kernels are compiled from (kernels, layout, registry, instantiation
    unit, generated tables, flags): unchanged while only host code of the ABI changes, so a
    profile of a kernel stays attributable to it."""
    h = hashlib.sha256(" ".join(NVCC_FLAGS).encode())
    for name in ("kernels.cuh", "layout.h", "registry.h", "ops_inst.cu", os.path.join("generated", "splines.h")):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def needs_build() -> bool:
    if not os.path.exists(OUT) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as f:
        return f.read().strip() != source_digest()


def _compile(args):
    cmd, stamp = args
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode == 0 and stamp:
        with open(stamp[0], "w") as f:
            f.write(stamp[1])
    return cmd, r.returncode, r.stdout + r.stderr


# the sources each object is compiled from (every unit includes the kernel headers)
UNIT_DEPS = {
    "interp": ["interp.cu", "kernels.cuh", "registry.h", "layout.h"],
    "ops": ["ops_inst.cu", "kernels.cuh", "registry.h", "layout.h"],
    "batch": ["batch_inst.cu", "kernels.cuh", "registry.h", "layout.h"],
}


def _unit_digest(cmd, kind) -> str:
    """Hash of an object's command line and the contents of what it is compiled from."""
    h = hashlib.sha256(" ".join(cmd).encode())
    for name in UNIT_DEPS[kind]:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    # the C header only reaches the ABI unit; every unit includes the generated tables
    for path in [GEN_HDR] + ([os.path.join(ROOT, "include", "interp.h")] if kind == "interp" else []):
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _job(cmd, obj, kind):
    """(cmd, (stamp path, digest)), or None when the object is up to date."""
    digest = _unit_digest(cmd, kind)
    stamp = obj + ".stamp"
    if os.path.exists(obj) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return None
    return cmd, (stamp, digest)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, jobs: int | None = None) -> str:
    if not force and not needs_build():
        return OUT
    objdir = os.path.join(BUILD, "obj")
    os.makedirs(objdir, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    extra = ["-Xptxas", "-v"] if ptxas_v else []
    jobsl = []
    objs = []

    def add(cmd, obj, kind):
        objs.append(obj)
        j = None if force else _job(cmd, obj, kind)
        if force:
            j = (cmd, (obj + ".stamp", _unit_digest(cmd, kind)))
        if j is not None:
            jobsl.append(j)

    o = os.path.join(objdir, "interp.o")
    add([nvcc(), *NVCC_FLAGS, *inc, "-c", os.path.join(CSRC, "interp.cu"), "-o", o], o, "interp")
    for name in spline_names():
        for part in range(N_PARTS):
            o = os.path.join(objdir, f"ops_{name}_{part}.o")
            add([nvcc(), *NVCC_FLAGS, *extra, *inc, f"-DINTERP_SPLINE={name}", f"-DINTERP_PART={part}",
                 "-c", os.path.join(CSRC, "ops_inst.cu"), "-o", o], o, "ops")
    o = os.path.join(objdir, "batch_3d.o")
    add([nvcc(), *NVCC_FLAGS, *extra, *inc, "-c", os.path.join(CSRC, "batch_inst.cu"), "-o", o], o, "batch")
    # the units of the large splines need several GB each: at most two of them run at a time
    big = [j for j in jobsl if any(k in " ".join(j[0]) for k in ("d4s", "voronoi2", "voronoi3"))]
    small = [j for j in jobsl if j not in big]
    logs = []
    with cf.ThreadPoolExecutor(max_workers=2) as exb, \
            cf.ThreadPoolExecutor(max_workers=max(1, (jobs or os.cpu_count() or 4) - 2)) as exs:
        futs = [exb.submit(_compile, j) for j in big] + [exs.submit(_compile, j) for j in small]
        for fu in futs:
            cmd, rc, out = fu.result()
            if verbose or rc != 0:
                logs.append(" ".join(cmd) + "\n" + out)
            if rc != 0:
                sys.stderr.write("\n".join(logs))
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if verbose:
        sys.stderr.write("\n".join(logs))
    tmp = OUT + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, OUT)
    with open(STAMP, "w") as f:
        f.write(source_digest())
    return OUT


PEAKS_SRC = os.path.join(CSRC, "peaks.cu")
PEAKS_OUT = os.path.join(BUILD, "libpeaks_b300.so")


def build_peaks(force: bool = False) -> str:
    """The microbenchmark library of csrc/peaks.cu (measured rooflines), rebuilt when its source
    or the flags change."""
    stamp = PEAKS_OUT + ".stamp"
    h = hashlib.sha256(" ".join(NVCC_FLAGS).encode())
    with open(PEAKS_SRC, "rb") as f:
        h.update(f.read())
    digest = h.hexdigest()
    if not force and os.path.exists(PEAKS_OUT) and os.path.exists(stamp) and open(stamp).read().strip() == digest:
        return PEAKS_OUT
    os.makedirs(BUILD, exist_ok=True)
    tmp = PEAKS_OUT + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *NVCC_FLAGS, "-shared", "-o", tmp, PEAKS_SRC])
    os.replace(tmp, PEAKS_OUT)
    with open(stamp, "w") as f:
        f.write(digest)
    return PEAKS_OUT


if __name__ == "__main__":
    build_peaks(force="--force" in sys.argv)
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv or "--ptxas-v" in sys.argv,
                ptxas_v="--ptxas-v" in sys.argv))
