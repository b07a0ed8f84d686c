"""Compile the C oracle into ``oracle/_build/liboracle.so`` with the host C compiler.

Test infrastructure only (see ``oracle/__init__.py``).  Plain ``-O2``: no vector
intrinsics, no ``-march=native``, so the same source gives the same bytes on x86_64 and
aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "dibr_oracle.c"), os.path.join(HERE, "inpaint2d_oracle.c")]


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources; return its path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        lib_mtime = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= lib_mtime for s in SOURCES if os.path.exists(s)):
            return LIB_PATH
    srcs = [s for s in SOURCES if os.path.exists(s)]
    tmp = LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True))
