"""Build libpcot.so in-tree for sm_103a (nvcc, one -gencode, parallel compiles).

Usage: python -m paper_1802_00166_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpcot.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC, "-I", BUILD]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpcot.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")) + [MODEL_INC])


MODEL_NPZ = os.path.join(PKG, "data", "picker.npz")
MODEL_INC = os.path.join(BUILD, "picker_model.inc")


def _model_include():
    """Write _build/picker_model.inc: the trained picker (MLP parameters,
    feature mean and standard deviation) as a C array, compiled into the
    library as every new handle's default model; no model when the trained
    file is absent."""
    if os.path.exists(MODEL_INC) and (not os.path.exists(MODEL_NPZ) or
                                      os.path.getmtime(MODEL_INC) >= os.path.getmtime(MODEL_NPZ)):
        return
    vals = []
    if os.path.exists(MODEL_NPZ):
        import numpy as np
        z = np.load(MODEL_NPZ)
        vals = [float(v) for v in np.concatenate([z["params"], z["feat_mean"], z["feat_std"]]).astype(np.float32)]
    lines = ["// Generated by build.py from data/picker.npz; do not edit.",
             f"static const int kPickerModelFloats = {len(vals)};",
             "static const float kPickerModel[] = {"]
    for i in range(0, len(vals), 6):
        lines.append("    " + ", ".join(f"{v!r}f" if v == v else "0.0f" for v in vals[i:i + 6]) + ",")
    if not vals:
        lines.append("    0.0f,")
    lines.append("};")
    tmp = MODEL_INC + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(tmp, MODEL_INC)


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + headers()):
        return obj, ""
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, extra=None) -> str:
    """Compile every CUDA/C++ source of the library and link libpcot.so."""
    os.makedirs(BUILD, exist_ok=True)
    _model_include()
    srcs = sources()
    if not force and not _stale(LIB, srcs + headers()):
        return LIB
    if force:
        for o in glob.glob(os.path.join(BUILD, "*.o")):
            os.remove(o)
    extra = list(extra or [])
    jobs = min(len(srcs), max(1, os.cpu_count() or 1))
    objs = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for obj, log in ex.map(lambda s: _compile(s, extra), srcs):
            objs.append(obj)
            if verbose and log:
                print(log, file=sys.stderr)
    cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
