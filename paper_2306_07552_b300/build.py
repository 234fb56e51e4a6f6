"""Builds the in-tree shared library libgx.so for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
SO = os.path.join(HERE, "libgx.so")
SOURCES = ["gx_api.cu", "gx_physics.cu", "gx_physics_store.cu", "gx_boxes.cu", "gx_boxes_store.cu", "gx_raster.cu", "gx_fused.cu", "gx_grid.cu", "gx_nsdf.cu",
           "gx_nsdf_train.cu", "gx_meshlets.cpp", "gx_store.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "gx.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, out: str = SO, defines=()) -> str:
    """Compiles libgx.so (or `out`, with extra -D `defines` for tuning runs)."""
    if out == SO and not defines and not force and not _stale():
        return SO
    cmd = (["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            *[f"-D{d}" for d in defines], "-o", out] + [os.path.join(CSRC, s) for s in SOURCES])
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd, cwd=HERE)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
