"""Build libplk.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2305_04318_b300.build [--force]

The shared library is written next to this file so that it travels with the
source tree; nothing is installed into site-packages.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libplk.so")
COUNTERS_LIB = os.path.join(HERE, "libplk_counters.so")
PROBE_SRC = os.path.join(HERE, "csrc_probe", "peak_probe.cu")
PROBE_LIB = os.path.join(HERE, "libplk_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.inc")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date(lib: str = None) -> bool:
    lib = lib or LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build_probe(force: bool = False) -> str:
    """libplk_probe.so: FMA-pipe throughput probe used by the benchmark."""
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    subprocess.run([os.environ.get("NVCC", "nvcc"), *ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC",
                    "-o", tmp, PROBE_SRC], check=True)
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def _build_lib(out: str, defines=(), verbose: bool = False) -> str:
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           *[f"-D{d}" for d in defines], "-I", INCLUDE, "-o", tmp, *sources(), "-lpthread"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    build_probe(force)
    if not force and up_to_date():
        return LIB
    return _build_lib(LIB, verbose=verbose)


def build_counters(force: bool = False, verbose: bool = False) -> str:
    """The diagnostic build with the trailing update's wait-cycle counters
    (-DPLK_PIPE_COUNTERS; plk_pipe_counters), next to the library."""
    if not force and up_to_date(COUNTERS_LIB):
        return COUNTERS_LIB
    return _build_lib(COUNTERS_LIB, defines=("PLK_PIPE_COUNTERS",), verbose=verbose)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
