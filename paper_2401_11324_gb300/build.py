"""Builds libbang.so, the C-ABI library of the search path, for sm_103a.

One translation unit, compiled in place with nvcc; the result lands next to
the sources (git-ignored) and is what the Python binding loads.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(CSRC, "libbang.so")
SOURCES = ["bang_api.cu", "link_probe.cu", "server.cu", "adc_table_tc.cu", "search_f32.cu",
           "search_bf16.cu", "search_exact.cu", "search_q8.cu", "autotune.cu", "build_graph.cu", "build_pq.cu", "ground_truth.cu",
           "build_shard.cu", "rerank.cu", "search_f32lazy.cu"]
HEADERS = ["search_kernel.cuh", "bang_internal.h", "adc_table_tc.h", "rerank.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [
        os.path.join(ROOT, "include", "bang.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=False):
    """Compile every translation unit in parallel, then link libbang.so."""
    if not force and not _stale():
        return LIB
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.append("-Xptxas=-v")
    objs, procs = [], []
    for f in SOURCES:
        obj = os.path.join(CSRC, os.path.splitext(f)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc(), *flags, "-c", os.path.join(CSRC, f), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((f, subprocess.Popen(cmd, cwd=CSRC)))
    failed = [f for f, p in procs if p.wait() != 0]
    if failed:
        raise RuntimeError("nvcc failed on %s" % ", ".join(failed))
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs], cwd=CSRC)
    os.replace(LIB + ".tmp", LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
