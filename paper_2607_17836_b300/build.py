"""Build libelpath.so (all CUDA sources for sm_103a) in place, next to this file."""
from __future__ import annotations

import glob
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libelpath.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(ROOT, "include", "elpath.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _inputs())


NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
FLAGS = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2"]


def nvcc_command(out: str, extra=()) -> list[str]:
    """One nvcc command compiling every source into `out` (sequential: slow)."""
    return [NVCC, *FLAGS, "-shared", "-o", out, *sources(), "-I", os.path.join(ROOT, "include"),
            "-lcufft", "-Xlinker", f"-rpath,{CUDA_HOME}/lib64", *extra]


def compile_commands(objdir: str, extra=()) -> list[tuple[str, list[str]]]:
    """(object, command) per source: compiled in parallel, each split over the
    host's cores (--split-compile)."""
    out = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        out.append((obj, [NVCC, *FLAGS, "--split-compile", "0", "-c", src, "-o", obj,
                          "-I", os.path.join(ROOT, "include"), *extra]))
    return out


def link_command(out: str, objs) -> list[str]:
    return [NVCC, *ARCH, "-shared", "-o", out, *objs, "-lcufft", "-Xlinker", f"-rpath,{CUDA_HOME}/lib64"]


def build_to(out: str, extra=(), verbose: bool = False) -> str:
    """Compile every source (in parallel) and link them into `out`."""
    with tempfile.TemporaryDirectory(prefix="elpath_build_") as objdir:
        jobs = compile_commands(objdir, extra)
        procs = []
        for obj, cmd in jobs:
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
        logs = [p.communicate()[0] for p in procs]
        for (obj, cmd), p, log in zip(jobs, procs, logs):
            if p.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + log)
            if verbose and log:
                print(log, file=sys.stderr)
        cmd = link_command(out, [obj for obj, _ in jobs])
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    return out


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not extra and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    build_to(tmp, extra, verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else ())
