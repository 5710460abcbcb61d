"""Build the FR-SG CUDA library in-tree: paper_2112_05946_gb300/libfrsg.so for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one shared
library.  Nothing is installed; the .so sits next to this file.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libfrsg.so")
PEAK_OUT = os.path.join(HERE, "libfrsg_peak.so")   # FMA throughput microbenchmark (not the scheme)
BUILD = os.path.join(HERE, "_build")

SOURCES = ["api.cu", "tables.cpp", "kern1d.cu", "kern1d_f32.cu", "kern1d_f64.cu", "kern2d.cu", "kmisc.cu", "noalloc.cu",
           "kadjoint.cu", "kadjoint_euler.cu", "kadjoint_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the FR-SG library needs the CUDA toolkit")
    return path


def _compile(src, verbose):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", INCLUDE,
           "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd[1:1] = ["-x", "cu"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    return obj, res.stderr


def _link(out, objs):
    tmp = out + ".tmp"
    cmd = [_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, out)


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t_out = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t_out for d in deps)


def build(verbose=False, force=False):
    """Compile every source for sm_103a and link libfrsg.so (and the FMA microbenchmark
    libfrsg_peak.so).  Returns the path of libfrsg.so."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(INCLUDE, "frsg.h")] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    peak_deps = [os.path.join(CSRC, "peak.cu"), os.path.join(INCLUDE, "frsg_peak.h")]
    main_stale = force or _stale(OUT, deps)
    peak_stale = force or _stale(PEAK_OUT, peak_deps)
    jobs = (SOURCES if main_stale else []) + (["peak.cu"] if peak_stale else [])
    if not jobs:
        return OUT
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = dict(zip(jobs, ex.map(lambda s: _compile(s, verbose), jobs)))
    if verbose:
        for _, log in results.values():
            sys.stderr.write(log)
    if main_stale:
        _link(OUT, [results[s][0] for s in SOURCES])
    if peak_stale:
        _link(PEAK_OUT, [results["peak.cu"][0]])
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
