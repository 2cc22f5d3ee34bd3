"""Build liblbpc.so in-tree for sm_103a with nvcc (no cmake, one gencode, parallel compilation).

    python -m paper_1709_04400_gb300.build [--force] [--verbose]
"""

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "liblbpc.so")
SOURCES = ["lbpc_api.cu", "lbpc_split.cu", "lbpc_fused.cu", "lbpc_batch_kernels.cu", "lbpc_batch_tiles.cu", "lbpc_batch.cu",
           "lbpc_static.cu", "lbpc_probe.cu"]
HEADERS = ["lbpc_device.cuh", "lbpc_dw.cuh", "lbpc_tile.cuh", "lbpc_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: install the CUDA toolkit or put nvcc on PATH")


def _inputs():
    return [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "lbpc.h")]


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force=False, verbose=False, extra_flags=()):
    """Compile every CUDA source of the library into liblbpc.so next to this file: one nvcc per
    translation unit, all at once, then one link."""
    if not force and up_to_date():
        return LIB
    nvcc = nvcc_path()
    obj_dir = os.path.join(PKG, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    # -prec-div=false -prec-sqrt=false: binary32 '/' and sqrtf take the approximate hardware forms
    # (about 2 ulp; the FP32 path is held to 1e-4). Binary64 arithmetic and the double-word type's
    # explicitly rounded intrinsics are not affected.
    flags = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "--threads", "0", "-prec-div=false", "-prec-sqrt=false",
             "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", os.path.join(ROOT, "include"), *extra_flags]
    objs, procs = [], []
    for f in SOURCES:
        o = os.path.join(obj_dir, f.replace(".cu", ".o"))
        cmd = [nvcc, *flags, "-c", "-o", o, os.path.join(CSRC, f)]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((f, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
        objs.append(o)
    failed = []
    for f, pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            failed.append(f"{f} ({pr.returncode}):\n{out}\n{err}")
        elif verbose and (out or err):
            print(out, err, flush=True)
    if failed:
        raise RuntimeError("nvcc failed: " + "\n".join(failed))
    link = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", LIB + ".tmp", *objs]
    if verbose:
        print(" ".join(link), flush=True)
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed ({r.returncode}):\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
