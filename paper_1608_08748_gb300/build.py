"""Build libmhd.so (the CUDA library behind include/mhd.h) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmhd.so")
SOURCES = ["mhd.cu", "mhd_noalloc.cu", "mhd_server.cu", "mhd_gravity.cu", "mhd_probe.cu"]
# FP32-bulk launchers: compiled separately with contraction on
SOURCES_F32 = ["mhd_f32.cu"]
HEADERS = ["mhd_device.cuh", "mhd_kernels.cuh", "mhd_runtime.cuh"]

# The FP64 path may contract a*b+c into FMAs (its kernels are bound by the FP64 pipe; contraction
# removes ~15 % of its instructions); it then agrees with the FP64 oracle to ~1e-14 relative L1.


def _stale(target: str = LIB) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(SRC, f) for f in SOURCES + SOURCES_F32 + HEADERS] + [os.path.join(ROOT, "include", "mhd.h")]
    return any(os.path.getmtime(d) > t for d in deps)


ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc] + ARCH + COMMON + extra + ["-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    return subprocess.Popen(cmd), cmd


LIB_CHECK = os.path.join(OUT_DIR, "libmhd_check.so")


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile the translation units in parallel and link libmhd.so (check=True: the index-checked
    libmhd_check.so, compiled with -DMHD_CHECK)."""
    target = LIB_CHECK if check else LIB
    if not force and not _stale(target):
        return target
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    tag = f".{os.getpid()}"
    jobs, objs = [], []
    for f in SOURCES + SOURCES_F32:
        obj = os.path.join(OUT_DIR, f.replace(".cu", tag + ".o"))
        # FP32 bulk: contraction and the hardware-approximate float division / square root (a few
        # ulp, far inside its 1e-4 target); its FP64 parts (chemistry, CFL) are unaffected.
        extra = (["--fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
                 if f in SOURCES_F32 else ["--fmad=true"])
        if check:
            extra = extra + ["-DMHD_CHECK"]
            obj = obj[:-2] + ".check.o"
        p, cmd = _compile(nvcc, os.path.join(SRC, f), obj, extra)
        if verbose:
            print(" ".join(cmd))
        jobs.append((p, cmd))
        objs.append(obj)
    for p, cmd in jobs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, cmd)
    tmp = target + f".tmp{os.getpid()}"
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcufft"]
    if verbose:
        print(" ".join(link))
    subprocess.run(link, check=True)
    for o in objs:
        os.remove(o)
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(build(force=True, verbose=True))
