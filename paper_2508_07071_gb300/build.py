"""Build libfkl.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

Every translation unit under csrc/ is compiled by nvcc in parallel, then
linked into paper_2508_07071_gb300/libfkl.so. Objects go to
paper_2508_07071_gb300/_build/. A build is skipped when the library is newer
than every source and header; otherwise only the objects whose source, or a
header they include (nvcc's dependency files), changed are compiled again.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfkl.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: plain float expressions are not contracted into multiply-adds;
# the kernels spell out each one they want (fmaf / fma.rn) and round every
# other operation where written (_rn intrinsics). The flag does not stop the
# assembler from fusing a packed f32x2 multiply into a packed add that
# consumes it, so the kernels never write that pair (see ops.cuh).
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-fvisibility=hidden", "-Xptxas", "-warn-spills", "--diag-suppress=177"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libfkl.so")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _all_inputs():
    out = list(sources())
    for d, _, files in os.walk(CSRC):
        out += [os.path.join(d, f) for f in files if f.endswith((".cuh", ".h"))]
    out.append(os.path.join(ROOT, "include", "fkl.h"))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _all_inputs())


def _deps(dep_file: str) -> list[str] | None:
    """Files an object was compiled from, from nvcc's dependency file (None
    when there is none)."""
    if not os.path.exists(dep_file):
        return None
    text = open(dep_file).read().replace("\\\n", " ")
    _, _, rest = text.partition(":")
    return [f for f in rest.split() if f]


def _object_current(src: str, obj: str, extra: list[str]) -> bool:
    """Whether `obj` is newer than its source, every header it included and
    the build script, and was compiled with the same extra flags."""
    dep, flags = obj[:-2] + ".d", obj[:-2] + ".flags"
    deps = _deps(dep)
    if deps is None or not os.path.exists(obj) or not os.path.exists(flags):
        return False
    if open(flags).read() != " ".join(extra):
        return False
    t = os.path.getmtime(obj)
    return all(os.path.exists(f) and os.path.getmtime(f) <= t for f in deps + [src, os.path.abspath(__file__)])


def _compile(src: str, extra: list[str], force: bool = False) -> str:
    obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
    if not force and _object_current(src, obj, extra):
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj,
           "-MD", "-MF", obj[:-2] + ".d"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-6000:]}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    with open(obj[:-2] + ".flags", "w") as f:
        f.write(" ".join(extra))
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile and link libfkl.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    if verbose:
        extra += ["-Xptxas", "-v"]
    srcs = sources()
    workers = min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, force), srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time
    t0 = time.time()
    path = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(f"built {path} in {time.time() - t0:.1f} s")
