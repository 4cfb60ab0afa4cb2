"""Compile the CPU oracle into oracle/libweno_oracle.so (test infrastructure).

Plain g++, no fused multiply-add (-ffp-contract=off) so the oracle gives the
same bits on x86-64 and AArch64 hosts.  build(variant="reversed") compiles
the same source with its final sums taken in the opposite order
(-DORA_REVERSED_SUMS=1) into libweno_oracle_rev.so: the same arithmetic
rounded differently, used to show how far a run amplifies rounding.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "weno_oracle.cpp")
LIB = os.path.join(HERE, "libweno_oracle.so")
VARIANTS = {None: ("libweno_oracle.so", []),
            "reversed": ("libweno_oracle_rev.so", ["-DORA_REVERSED_SUMS=1"])}


def build(force: bool = False, variant=None) -> str:
    name, defs = VARIANTS[variant]
    lib = os.path.join(HERE, name)
    deps = [SRC, os.path.join(HERE, "weno_oracle.h"), os.path.abspath(__file__)]
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in deps)):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function"] + defs + [SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False):
    return [build(force, v) for v in VARIANTS]


if __name__ == "__main__":
    for p in build_all(force=True):
        print(p)
