"""Builds the STEV CUDA library (libstev.so) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libstev.so")
PEAKS = os.path.join(HERE, "alu_peaks")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cuh", ".h"))] + [
        os.path.join(HERE, "..", "include", "stev.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    deps = _sources()
    if force or _stale(LIB, deps):
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
               "--expt-relaxed-constexpr", "-Xptxas", "-v" if verbose else "-O3",
               "-o", tmp, os.path.join(CSRC, "stev_capi.cu"),
               os.path.join(CSRC, "stev_server.cu"), os.path.join(CSRC, "stev_spec.cu"),
               os.path.join(CSRC, "stev_lm.cu"), os.path.join(CSRC, "stev_multiphase.cu"),
               "-lnvrtc"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed building libstev.so")
        if verbose:
            sys.stderr.write(r.stderr)
        os.replace(tmp, LIB)
    src = os.path.join(CSRC, "alu_peaks.cu")
    if force or _stale(PEAKS, [src]):
        tmp = PEAKS + ".%d.tmp" % os.getpid()
        subprocess.check_call([NVCC, *ARCH, "-O3", "-lineinfo", "-o", tmp, src])
        os.replace(tmp, PEAKS)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
