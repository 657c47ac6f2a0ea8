"""Build the CPU oracle (plain C) into oracle/liboracle.so with gcc.

The oracle is test infrastructure; building it is part of the package build
so that the tests and the benchmark's CPU-baseline leg can load it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle_symbolic.c", "selinv_oracle.c"]
DEPS = SOURCES + ["oracle_numeric.inc"]
TARGET = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = [os.path.join(HERE, s) for s in DEPS]
    if (not force and os.path.exists(TARGET)
            and os.path.getmtime(TARGET) >= max(os.path.getmtime(d) for d in deps)):
        return TARGET
    tmp = TARGET + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-pthread", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
