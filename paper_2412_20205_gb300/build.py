"""Build libigamg.so (the C-ABI library) in-tree for sm_103a with plain nvcc/g++.

Translation units are compiled in parallel; the result is
``paper_2412_20205_gb300/libigamg.so``.  No torch headers are involved.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libigamg.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
           "--expt-relaxed-constexpr"]
SOURCES = ["kernels.cu", "api.cu", "noalloc.cu", "cnn.cu", "tail.cu", "refine.cu", "general.cu", "host_setup.cpp",
           "general_setup.cpp"]


def _cmd(src, obj):
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        return [NVCC] + ARCH + CUFLAGS + ["-c", path, "-o", obj]
    return ["g++", "-O2", "-fPIC", "-std=c++17", "-I" + INCLUDE, "-c", path, "-o", obj]


def build(verbose=False, force=False):
    os.makedirs(BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC))
    newest_src = max(newest_src, os.path.getmtime(os.path.join(INCLUDE, "igamg.h")),
                     os.path.getmtime(__file__))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > newest_src:
        return LIB
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.rsplit(".", 1)[0] + ".o")
        objs.append(obj)
        cmd = _cmd(src, obj)
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out = p.communicate()[0].decode()
        if p.returncode != 0:
            failed.append((src, out))
        elif verbose and out.strip():
            print(out)
    if failed:
        raise RuntimeError("build failed:\n" + "\n".join(f"== {s}\n{o}" for s, o in failed))
    link = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.run(link, check=True)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
