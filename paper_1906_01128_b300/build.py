"""Build ``libdc.so`` (the C-ABI library) in place with nvcc for sm_103a."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
SO = os.path.join(HERE, "libdc.so")
SOURCES = ["kernels.cu", "plan.cpp", "runtime.cpp", "transfer.cpp", "step.cpp", "tune.cpp", "server.cpp", "arena.cpp", "spans.cpp", "static_scratch.cu", "trace.cpp", "debug.cpp", "partition.cpp"]
HEADERS = ["internal.hpp", "pool.hpp", "trace.hpp"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(HERE, "..", "include", "dc.h"))
    files.append(os.path.abspath(__file__))
    return files


def needs_build() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return SO
    cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
           "-shared", "-Xcompiler", "-fPIC,-O3,-pthread,-Wall,-fvisibility=hidden", "-cudart", "shared",
           "-Xlinker", "-rpath,/usr/local/cuda/lib64",
           "-o", SO + ".tmp"] + [os.path.join(CSRC, f) for f in SOURCES] + ["-lpthread"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(SO + ".tmp", SO)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(SO)
