"""Build the native parts of the package in-tree.

* ``libfbp.so``          -- the CUDA library behind ``include/fbp.h``, compiled
                            for sm_103a only (``-gencode arch=compute_103a,code=sm_103a``);
* ``libfbp_checked.so``  -- the same sources with ``-DFBP_CHECKED``: every
                            interpolation index is range-checked in the kernel
                            and a violation is recorded in the device status
                            word instead of being read (used by a GPU test);
* ``libphantom.so``      -- the host C input generator.

Translation units compile in parallel; no cmake.  Outputs are git-ignored.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")

CU_SOURCES = ["runtime.cu", "filter.cu", "backproject.cu", "forward.cu", "fbp_api.cu", "noalloc.cu", "sap.cu",
              "bp_texture.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers_mtime() -> float:
    paths = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, obj: str, defines: list[str]) -> None:
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, *defines,
           "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")


def build_cuda(name: str = "libfbp.so", defines: list[str] | None = None,
               force: bool = False, jobs: int | None = None) -> str:
    defines = defines or []
    out = os.path.join(HERE, name)
    srcs = [os.path.join(CSRC, s) for s in CU_SOURCES]
    newest = max([os.path.getmtime(s) for s in srcs] + [_headers_mtime(),
                                                       os.path.getmtime(__file__)])
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tag = name.replace(".so", "")
    bdir = os.path.join(BUILD, tag)
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in CU_SOURCES]
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(CU_SOURCES), os.cpu_count() or 4)) as ex:
        futs = [ex.submit(_compile, s, o, defines) for s, o in zip(CU_SOURCES, objs)]
        for f in futs:
            f.result()
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> list[str]:
    from . import phantoms
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build_cuda, "libfbp.so", [], force)
        b = ex.submit(build_cuda, "libfbp_checked.so", ["-DFBP_CHECKED"], force)
        outs = [a.result(), b.result()]
    outs.append(phantoms.build(force=force))
    return outs


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    from paper_2505_13955_gb300 import build as _b
    for p in _b.build_all(force="--force" in sys.argv):
        print(p)
