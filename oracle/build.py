"""Compile the oracle's C sources into a shared library (test infrastructure).

Plain gcc, no vendor flags, so the same source builds on x86-64 and aarch64.
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build", platform.machine())   # one per host architecture
LIB_PATH = os.path.join(BUILD_DIR, "libndft_oracle.so")
SOURCES = [os.path.join(HERE, "ndft.c")]


def build(force: bool = False) -> str:
    """Build libndft_oracle.so if missing or older than its sources."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SOURCES)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp] + SOURCES + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
