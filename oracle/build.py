"""Compile the FP64 reference GEMM (``gemm_ref.c``) into a shared library.

Test infrastructure only: the GPU library never loads what this builds.
Plain gcc, no vector extensions and ``-ffp-contract=off`` so that every
multiply and add rounds once in FP64, identically on x86-64 and AArch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SRC = os.path.join(HERE, "gemm_ref.c")


def _stale():
    return (not os.path.exists(LIB_PATH)) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC)


def build_oracle(force=False, openmp=True):
    """Build ``_build/liboracle.so`` if missing or older than the source."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    cmd = base[:1] + (["-fopenmp"] if openmp else []) + base[1:]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0 and openmp:
        # no libgomp on this host: serial oracle, same arithmetic
        res = subprocess.run(base, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + res.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def build_variant(src_text, out_path, openmp=False):
    """Compile a modified copy of the oracle source (used by the mutation
    tests that show the pins catch planted mistakes)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    cmd = ["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
           src, "-o", out_path, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("variant build failed:\n" + res.stderr)
    return out_path


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
