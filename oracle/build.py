"""Build the FP64 CPU oracle (test infrastructure) into oracle/_build/liboracle.so
(the renderer in gs_oracle.cpp, the level-of-detail hierarchy in
gs_lod_oracle.cpp).

Plain g++, IEEE double arithmetic (no fast-math, no FMA contraction flags);
OpenMP for the loops over Gaussians and tiles (results do not depend on the
thread count).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "gs_oracle.cpp"), os.path.join(HERE, "gs_lod_oracle.cpp")]
OUT = os.path.join(HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    if (not force and os.path.exists(OUT)
            and all(os.path.getmtime(OUT) >= os.path.getmtime(src) for src in SRCS)):
        return OUT
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           "-Wall", "-Wextra", "-o", tmp, *SRCS]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
