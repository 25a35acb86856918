"""Build libgs.so (the CUDA rasterizer and its C ABI) for sm_103a.

Each .cu under csrc/ is compiled with nvcc for `-gencode arch=compute_103a,
code=sm_103a` and linked into paper_2607_14481_b300/_build/libgs.so (in tree,
so it travels with the repository snapshot).  Rebuilds only when a source or
header is newer than the library.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgs.so")
ROOT = os.path.dirname(HERE)
ARCH = "103a"

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-lineinfo",
    f"-gencode=arch=compute_{ARCH},code=sm_{ARCH}",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
    "-DGS_BUILT_ARCH=1030",
    "--expt-relaxed-constexpr",
]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))) \
        + [os.path.join(ROOT, "include", "gs.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, jobs: int = 8) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    objs, procs = [], []
    for src in _sources():
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        if len(procs) >= jobs:
            _wait(procs, verbose)
            procs = []
    _wait(procs, verbose)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run([nvcc, "-shared", f"-gencode=arch=compute_{ARCH},code=sm_{ARCH}", "-o", tmp, *objs,
                    "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


def _wait(procs, verbose):
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            sys.stderr.write(text)
            raise RuntimeError("nvcc failed on " + os.path.basename(src))
        if verbose and text.strip():
            sys.stderr.write(text)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
