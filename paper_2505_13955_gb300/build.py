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

FILTER_UNITS = [f"filter_{fam}_{dt}.cu" for fam in ("plain", "stream", "batched")
                for dt in ("f32", "f16", "bf16")]
CU_SOURCES = ["runtime.cu", "filter.cu", *FILTER_UNITS, "backproject.cu", "forward.cu", "fbp_api.cu",
              "noalloc.cu", "sap.cu", "bp_texture.cu", "probe.cu", "host_pipeline.cu", "bp_staged.cu",
              "bp_staged_batch.cu"]
# only these translation units read FBP_CHECKED; the checked twin shares every other object
CHECKED_SOURCES = ["backproject.cu"]
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


def _objects(tag: str, sources: list[str], defines: list[str], ex) -> list:
    bdir = os.path.join(BUILD, tag)
    os.makedirs(bdir, exist_ok=True)
    out = []
    for src in sources:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        out.append((obj, ex.submit(_compile, src, obj, defines)))
    return out


def _link(name: str, objs: list[str]) -> str:
    out = os.path.join(HERE, name)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build_cuda(force: bool = False, jobs: int | None = None) -> list[str]:
    """libfbp.so and libfbp_checked.so: every translation unit compiled once
    (in parallel), CHECKED_SOURCES a second time with -DFBP_CHECKED."""
    names = ("libfbp.so", "libfbp_checked.so")
    srcs = [os.path.join(CSRC, s) for s in CU_SOURCES]
    newest = max([os.path.getmtime(s) for s in srcs] + [_headers_mtime(), os.path.getmtime(__file__)])
    outs = [os.path.join(HERE, n) for n in names]
    if not force and all(os.path.exists(o) and os.path.getmtime(o) >= newest for o in outs):
        return outs
    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        # the longest units first, so the pool stays busy
        order = sorted(CU_SOURCES, key=lambda s: (not s.startswith("filter_"), s))
        plain = dict(_objects("libfbp", order, [], ex))
        checked = dict(_objects("libfbp_checked", CHECKED_SOURCES, ["-DFBP_CHECKED"], ex))
        for fut in list(plain.values()) + list(checked.values()):
            fut.result()
    objs = [os.path.join(BUILD, "libfbp", s.replace(".cu", ".o")) for s in CU_SOURCES]
    objs_checked = [os.path.join(BUILD, "libfbp_checked", s.replace(".cu", ".o")) if s in CHECKED_SOURCES
                    else o for s, o in zip(CU_SOURCES, objs)]
    return [_link(names[0], objs), _link(names[1], objs_checked)]


def build_all(force: bool = False) -> list[str]:
    from . import phantoms
    outs = build_cuda(force=force)
    outs.append(phantoms.build(force=force))
    return outs


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    from paper_2505_13955_gb300 import build as _b
    for p in _b.build_all(force="--force" in sys.argv):
        print(p)
