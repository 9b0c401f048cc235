"""Build librdg.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked with the CUDA runtime.  The
result lands in paper_1912_06221_gb300/_lib/librdg.so (git-ignored).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "librdg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object name, extra defines): the hot-path kernels build once per order/precision
SOURCES = [("refops.cpp", "refops", []), ("api.cpp", "api", []), ("rhs_dispatch.cpp", "rhs_dispatch", []),
           ("setup.cu", "setup", []), ("rhs_static.cu", "rhs_static", []), ("batch.cpp", "batch", []),
           ("measure.cu", "measure", []), ("halo.cu", "halo", []),
           ("batch_kernel.cu", "batch_kernel", [])]
for _n in range(1, 7):
    for _t, _tag in (("float", "f"), ("double", "d")):
        SOURCES.append(("rhs_order.cu", "rhs_%s%d" % (_tag, _n),
                        ["-DRDG_ORDER=%d" % _n, "-DRDG_REAL=%s" % _t, "-DRDG_TAG=%s" % _tag,
                         "-DRDG_TAG_IS_F=%d" % (_tag == "f")]))


def nvcc_path():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH, "-c", src, "-o", obj, *extra]
    if src.endswith(".cpp"):
        cmd = [nvcc, "-std=c++17", "-O2", "-x", "c++", "-Xcompiler", "-fPIC", "-c", src, "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stderr


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False) -> str:
    nvcc = nvcc_path()
    os.makedirs(OUT, exist_ok=True)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(HERE, "..", "include", "rdg.h")]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(d) for d in deps)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    objs = []
    jobs = []
    workers = max(1, min(len(SOURCES), os.cpu_count() or 1))
    # longest units first so the parallel build ends early
    order = sorted(SOURCES, key=lambda x: -int(x[1][-1]) if x[1][-1].isdigit() else 0)
    with ThreadPoolExecutor(max_workers=workers) as ex:
        for s, name, defs in order:
            obj = os.path.join(OUT, name + ".o")
            objs.append(obj)
            jobs.append((name, ex.submit(_compile, nvcc, os.path.join(SRC, s), obj, extra + defs)))
        for s, j in jobs:
            msg = j.result()
            if verbose and msg:
                print("==", s, "\n", msg, file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv, force=True))
