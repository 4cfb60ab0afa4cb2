"""Compile the CPU oracle into oracle/libweno_oracle.so (test infrastructure).

Plain g++, no fused multiply-add (-ffp-contract=off) so the oracle gives the
same bits on x86-64 and AArch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "weno_oracle.cpp")
LIB = os.path.join(HERE, "libweno_oracle.so")


def build(force: bool = False) -> str:
    deps = [SRC, os.path.join(HERE, "weno_oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
