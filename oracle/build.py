"""Compile the CPU oracle (rac_oracle.c) into oracle/liboracle.so with gcc.

Test infrastructure only: the oracle is built beside the product so that the
tests can run, never linked into it."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rac_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-Wall", "-Wextra", "-o", tmp, src])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
