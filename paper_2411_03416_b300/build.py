"""Builds the CUDA library libpgvimp.so in-tree for sm_103a.

Each state dimension's kernels live in their own translation unit so that
nvcc runs them in parallel.  The library lands in
paper_2411_03416_b300/_build/libpgvimp.so.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpgvimp.so")
ROOT = os.path.dirname(HERE)

SOURCES = ["pgvimp_api.cu", "pgvimp_noalloc.cu", "pgvimp_server.cu", "k4_lane_df.cu", "k4_lane_f32.cu",
           "k4_lane_f64.cu"] + [f"k{n}_{part}.cu" for n in (14, 6, 4)
                               for part in ("iter_df", "iter_f32", "cta_f32", "iter_f64", "cta_f64",
                                            "cta_df", "aux", "aux_df", "rows")]
HEADERS = ["pgvimp_device.cuh", "pgvimp_dfx.cuh", "pgvimp_kernels.cuh", "pgvimp_cr.cuh", "pgvimp_crw.cuh",
           "pgvimp_lane.cuh", "pgvimp_plan.h",
           "pgvimp_launch.h", "pgvimp_internal.h", "pgvimp_pool.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
EXTRA_FLAGS = {}   # per-unit extra nvcc flags
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _headers_of(src: str):
    """The headers a translation unit includes (directly or through another)."""
    base = ["pgvimp_plan.h"]
    if src.startswith("k"):
        base += ["pgvimp_device.cuh", "pgvimp_kernels.cuh", "pgvimp_launch.h"]
        if "_cta_" in src:
            base += ["pgvimp_cr.cuh", "pgvimp_crw.cuh", "pgvimp_dfx.cuh"]
        if "_lane_" in src:
            base += ["pgvimp_lane.cuh", "pgvimp_dfx.cuh"]
    elif src == "pgvimp_api.cu":
        base += ["pgvimp_device.cuh", "pgvimp_launch.h", "pgvimp_internal.h"]
    elif src == "pgvimp_server.cu":
        base += ["pgvimp_internal.h", "pgvimp_pool.h"]
    elif src == "pgvimp_noalloc.cu":
        base += ["pgvimp_device.cuh"]
    else:
        base = list(HEADERS)
    return base


def _deps_mtime(src: str):
    files = [os.path.join(CSRC, h) for h in _headers_of(src)] + [os.path.join(ROOT, "include", "pgvimp.h")]
    if src in EXTRA_FLAGS:
        files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, "obj", src.replace(".cu", ".o"))
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), _deps_mtime(src)):
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *EXTRA_FLAGS.get(src, []), "-c", s, "-o", o]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((src, cmd))

    def run(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for src, r in ex.map(run, jobs):
            if verbose or r.returncode != 0 or ptxas_info:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}")
    objs = [os.path.join(OUT, "obj", s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of libpgvimp.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
