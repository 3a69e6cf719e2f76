"""Build of libdartray.so (CUDA, sm_103a) in-tree.

The translation units (the CUDA sweep, the marcher for 4-16 wavelengths and
the host grid builder) compile in parallel and link into
paper_1709_03802_gb300/_build/libdartray.so.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdartray.so")
SOURCES = [os.path.join(CSRC, "dartray.cu"), os.path.join(CSRC, "march_wide.cu"), os.path.join(CSRC, "grid_host.cpp")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
    [os.path.join(os.path.dirname(HERE), "include", "dartray.h")]


def nvcc():
    cand = os.environ.get("NVCC") or os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in DEPS)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    flags = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC"]
    # extra compiler flags, e.g. -DDARTRAY_MARCH_MIN_BLOCKS=6 (tuning builds)
    flags += os.environ.get("DARTRAY_NVCC_FLAGS", "").split()
    if verbose:
        flags.append("-Xptxas=-v")
    # translation units in parallel, then one link
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.basename(src) + f".{os.getpid()}.o")
        cmd = [nvcc()] + flags + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    bad = [p.args for p in procs if p.wait() != 0]
    if bad:
        raise subprocess.CalledProcessError(1, bad[0])
    subprocess.check_call([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs)
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
