"""Builds libproxybdpt.so for sm_103a in-tree (paper_2503_23412_gb300/_build).

Each translation unit is compiled in parallel with nvcc, then linked as a
shared library. Host code only uses portable C++17, so the same build runs on
x86-64 and on Arm (Grace) hosts.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libproxybdpt.so")
ROOT = os.path.dirname(HERE)
HEADERS = [os.path.join(ROOT, "include", "proxybdpt.h")] + [
    os.path.join(CSRC, f) for f in ("pb_device.cuh", "pb_kernels.h", "pb_bvh.h", "pb_ctx.h", "pb_estimator.cuh",
                                    "pb_mlp.cuh", "pb_entry.cuh", "pb_recip_long.cuh")]
UNITS = ["pb_api.cu", "pb_light.cu", "pb_recip.cu", "pb_recip_long.cu", "pb_recip_long_count.cu", "pb_wavefront.cu",
         "pb_eye.cu", "pb_learn.cu", "pb_noalloc.cu", "pb_mlp.cu", "pb_probe.cu", "pb_bvh.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    procs, objs = [], []
    for u in UNITS:
        src = os.path.join(CSRC, u)
        obj = os.path.join(BUILD, u + ".o")
        objs.append(obj)
        if not force and not _stale(obj, [src] + HEADERS):
            continue
        cmd = [nv] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
        if u.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        cmd += list(extra)
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for u, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(u)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    if force or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nv] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
