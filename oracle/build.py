"""Compile the FastMuyGPs oracle (plain C11, FP64, -ffp-contract=off) into
oracle/_liboracle.so.  Test infrastructure only: the CUDA library never uses it."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = [os.path.join(HERE, "fmgp_oracle.c"), os.path.join(HERE, "oracle_core.h")]
TARGET = os.path.join(HERE, "_liboracle.so")


def needs_build() -> bool:
    if not os.path.exists(TARGET):
        return True
    t = os.path.getmtime(TARGET)
    return any(os.path.getmtime(s) > t for s in SOURCES)


def build_variant(defines, target):
    """Compile the oracle with extra -D macros into `target` (mutation tests)."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared"] + [f"-D{m}" for m in defines] + ["-o", target, SOURCES[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    return target


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = TARGET + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, SOURCES[0], "-lm"]
        subprocess.run(cmd, check=True, cwd=HERE)
        os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
