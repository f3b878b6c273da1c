"""Build the in-tree shared library ``_lib/liblamg_b300.so`` for sm_103a.

CUDA sources go through nvcc with ``-gencode arch=compute_103a,code=sm_103a -lineinfo``;
the host-setup C++ goes through nvcc's host compiler with ``-ffp-contract=off`` so that the
setup's floating-point decisions are evaluated exactly as written. The CUDA runtime is
linked statically; the library exports only the ``lamg_*`` C ABI of ``include/lamg.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
SO = os.path.join(OUT_DIR, "liblamg_b300.so")
BUILD_DIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-I", INC, "-I", CSRC, "-Xcompiler", "-fPIC",
          "-Xcompiler", "-ffp-contract=off"]
CU_FLAGS = ARCH + ["-lineinfo", "--expt-relaxed-constexpr"] + COMMON


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _stale(srcs: list[str]) -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    deps.append(os.path.join(INC, "lamg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    srcs = sources()
    if not force and not _stale(srcs):
        return SO
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        flags = list(CU_FLAGS)
        if src.endswith(".cu") and ptxas_v:
            flags += ["-Xptxas", "-v"]
        cmd = [nvcc, "-c", src, "-o", obj] + flags
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "c++", "-c", src, "-o", obj] + COMMON
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
        if verbose or ptxas_v:
            sys.stderr.write(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
