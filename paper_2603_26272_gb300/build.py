"""Build libweno.so (CUDA, sm_103a) in-tree.

nvcc compiles each translation unit in parallel and links one shared library
with the CUDA runtime linked statically, so the library only needs the
driver (libcuda) at run time.  IEEE division and square root are kept (no
--use_fast_math): the FP64 path must match the CPU oracle to 1e-12.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libweno.so")
SOURCES = ["weno_kernels.cu", "weno_orders.cu", "weno_api.cu", "weno_noalloc.cu", "weno_engine.cu",
           "weno_peak.cu"]
HEADERS = ["weno_device.cuh", "weno_tiles.cuh", "weno_tiles1d.cuh", "weno_internal.h"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else "nvcc"


def _flags(verbose=False):
    f = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2",
         "-I", os.path.join(ROOT, "include")]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def build(force=False, verbose=False):
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "weno.h"))
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for s in SOURCES:
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc()] + _flags(verbose) + ["-c", os.path.join(CSRC, s), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    logs = []
    ok = True
    for cmd, p in procs:
        out, _ = p.communicate()
        logs.append(out.decode(errors="replace"))
        if p.returncode != 0:
            ok = False
    if verbose or not ok:
        sys.stderr.write("\n".join(logs))
    if not ok:
        raise RuntimeError("nvcc failed")
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run([nvcc(), "-shared", ARCH, "-cudart", "static", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
