"""Build libcg.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")

SOURCES = ["cg_kernels.cu", "cg_scan_tma.cu", "cg_scan_level.cu", "cg_noalloc.cu", "cg_mlp.cu", "cg_scan_pitched.cu",
           "cg_devops_kernels.cu", "cg_host.cpp", "cg_batch.cpp", "cg_serve.cpp", "cg_pitched.cpp",
           "cg_devops.cpp", "cg_snapshot.cpp"]


def _cmd_compile(src: str, obj: str, host_flags=()) -> list[str]:
    extra = os.environ.get("CG_NVCC_FLAGS", "").split()
    for f in host_flags:  # one at a time: nvcc splits a flag list at commas
        extra += ["-Xcompiler", f]
    common = [NVCC, "-c", "-std=c++17", "-O3", "-Xcompiler", "-fPIC,-Wall"] + extra + [
              "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-o", obj]
    if src.endswith(".cu"):
        return common + ARCH + ["-lineinfo", "-Xptxas", "-v" if os.environ.get("CG_PTXAS_V") else "-O3",
                                src]
    return common + [src]


def build(verbose: bool = False, out: str = LIB, obj_dir: str = OUT_DIR,
          host_flags=()) -> str:
    """Compile every source in parallel, then link the shared library.
    host_flags (for the host compiler, each without commas) and another
    output path give instrumented builds, e.g. with the sanitizers."""
    OUT = obj_dir
    os.makedirs(OUT, exist_ok=True)
    procs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT, os.path.splitext(s)[0] + ".o")
        objs.append(obj)
        cmd = _cmd_compile(src, obj, host_flags)
        if verbose:
            print(" ".join(cmd))
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True)))
    failed = []
    for cmd, p in procs:
        log, _ = p.communicate()
        if log and (verbose or p.returncode):
            sys.stderr.write(log)
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("libcg compile failed:\n" + "\n".join(failed))
    tmp = out + ".tmp"
    link = [NVCC, "-shared", "-o", tmp] + ARCH + objs + ["-Xcompiler", "-fPIC"]
    for f in host_flags:
        link += ["-Xcompiler", f]
    subprocess.run(link, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
