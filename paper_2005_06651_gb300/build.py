"""Build libvl2mhd.so and its value-safe twin libvl2mhd_vs.so (sm_103a) in-tree with nvcc.

The translation units compile in parallel; the shared library links the CUDA runtime dynamically so
that it shares the runtime (and the primary context) that PyTorch loads.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libvl2mhd.so")
# The value-safe parity build: IEEE division and square root in place of the Newton forms, and no FMA
# contraction (-fmad=false), for bitwise mirror-symmetric results (Sec. 3.3.5).  Same sources and ABI.
LIB_VALUE_SAFE = os.path.join(BUILD, "libvl2mhd_vs.so")
SOURCES = ["vl2_api.cu", "vl2_kernels.cu", "vl2_flux.cu", "vl2_adjoint.cu", "vl2_noalloc.cu", "vl2_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
VARIANTS = {LIB: ("", []), LIB_VALUE_SAFE: ("vs_", ["-fmad=false", "-DVL2_VALUE_SAFE"])}


def nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or cand)


def cuda_lib_dir():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        p = os.path.join(home, sub)
        if os.path.isdir(p):
            return p
    return os.path.join(home, "lib64")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "vl2mhd.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, libs=(LIB, LIB_VALUE_SAFE)) -> str:
    """Compile every translation unit of each requested library (all in parallel) and link them; returns the
    path of the default library."""
    os.makedirs(BUILD, exist_ok=True)
    todo = [lib for lib in libs if force or not os.path.exists(lib) or os.path.getmtime(lib) < _deps()]
    if not todo:
        return LIB
    base = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-Xptxas", "-v"]
    procs, objs = [], {lib: [] for lib in todo}
    for lib in todo:
        prefix, extra = VARIANTS[lib]
        for src in SOURCES:
            obj = os.path.join(BUILD, prefix + src.replace(".cu", ".o"))
            objs[lib].append(obj)
            log = open(obj + ".log", "w")
            cmd = [nvcc()] + base + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
            procs.append((subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), cmd, log, obj))
    failed = []
    for p, cmd, log, obj in procs:
        rc = p.wait()
        log.close()
        if rc != 0:
            failed.append((cmd, open(obj + ".log").read()))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + out for c, out in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    for lib in todo:
        tmp = lib + ".tmp%d" % os.getpid()
        link = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs[lib] + \
            ["-Xlinker", "-rpath," + cuda_lib_dir()]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout + r.stderr)
        os.replace(tmp, lib)
        if verbose:
            for obj in objs[lib]:
                sys.stdout.write(open(obj + ".log").read())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
