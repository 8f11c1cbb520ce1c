"""Builds libapip.so in-tree for sm_103a with nvcc (no cmake, no torch
extension machinery): each translation unit is compiled in parallel and the
objects are linked with the static CUDA runtime.  build(checked=True) builds the
bounds-checked variant libapip_checked.so (-DAPIP_CHECK_BOUNDS, objects in a
folder of their own); the binding loads it when APIP_LIBRARY names it."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libapip.so")
OUT_DIR_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libapip_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["apip.cu", "kernels_atoms.cu", "kernels_ace_f32.cu", "kernels_ace_f64.cu", "kernels_ace3_f32.cu",
           "kernels_ace3_f64.cu", "ace_tables.cpp", "apip_static.cu", "kernels_mlp.cu", "peak_probe.cu", "kernels_train_tc.cu"]
HEADERS = ["apip_internal.h", "device_common.cuh", "kernels.h", "ace_device.cuh", "ace_pool.cuh", "ace_stream.cuh",
           "gaunt_layout.h", "tc_common.cuh"]


def _flags(checked=False):
    return (["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
             "-I" + os.path.join(ROOT, "include"), "-I" + CSRC] + ARCH + (["-DAPIP_CHECK_BOUNDS"] if checked else []))


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(ROOT, "include", "apip.h")] + [os.path.join(CSRC, h) for h in HEADERS]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, ptxas_v=False, checked=False):
    """Compile and link libapip.so (checked: libapip_checked.so) if any source is
    newer than it; return its path."""
    out_dir, lib = (OUT_DIR_CHECKED, LIB_CHECKED) if checked else (OUT_DIR, LIB)
    os.makedirs(out_dir, exist_ok=True)
    jobs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
        if _stale(obj, path) or ptxas_v:
            cmd = [NVCC] + _flags(checked) + ["-c", path, "-o", obj]
            if src.endswith(".cpp"):
                cmd[1:1] = ["-x", "cu"]
            if ptxas_v and src.endswith(".cu"):
                cmd.append("-Xptxas=-v")
            jobs.append((src, cmd))

    def run(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for src, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}")
    objs = [os.path.join(out_dir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    if jobs or not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", lib] + objs + ["-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of " + os.path.basename(lib) + " failed")
    return lib


if __name__ == "__main__":
    print(build(verbose=True, ptxas_v="-v" in sys.argv, checked="--checked" in sys.argv))
