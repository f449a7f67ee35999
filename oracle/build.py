"""Build the C part of the oracle (liboracle.so, in-tree) with gcc.

TEST INFRASTRUCTURE ONLY: see oracle/__init__.py.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rpb_oracle.c")
GEN = os.path.join(HERE, "wall_image.c")
MCMC = os.path.join(HERE, "mcmc.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than its sources; return its path."""
    if not force and os.path.exists(LIB):
        mt = os.path.getmtime(LIB)
        if all(mt >= os.path.getmtime(f) for f in (SRC, GEN, MCMC)):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, SRC, MCMC, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
