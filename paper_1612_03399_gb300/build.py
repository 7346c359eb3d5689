"""In-tree build of the CUDA library (libibm_gb300.so) for sm_103a.

Each .cu translation unit is compiled by nvcc in parallel, then linked into
one shared library under paper_1612_03399_gb300/_build/.  The library links
the CUDA runtime statically, so loading it needs no GPU.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libibm_gb300.so")
SOURCES = ["ibm_host.cu", "k_mls.cu", "k_mls64.cu", "k_tile.cu", "k_force.cu", "k_adjoint.cu", "k_taylor.cu",
           "ibm_noalloc.cu", "ibm_gts.cu", "k_pc.cu", "ibm_flow.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ["../../include/ibm.h"]:
        p = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(p):
            h.update(name.encode())
            h.update(open(p, "rb").read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


# the sources each profiled kernel is compiled from (for per-kernel digests)
KERNEL_SOURCES = {
    "marker": ["k_mls.cu", "mls_closed_form.cuh", "bulk_copy.cuh", "ibm_internal.cuh"],
    "marker_p128": ["k_mls.cu", "mls_closed_form.cuh", "bulk_copy.cuh", "ibm_internal.cuh"],
    "clear": ["k_mls.cu", "mls_closed_form.cuh", "bulk_copy.cuh", "ibm_internal.cuh"],
    "forcing": ["k_mls.cu", "mls_closed_form.cuh", "bulk_copy.cuh", "ibm_internal.cuh"],
    "body_marker": ["k_mls.cu", "mls_closed_form.cuh", "bulk_copy.cuh", "ibm_internal.cuh"],
    "force": ["k_force.cu", "force_elems.cuh", "bulk_copy.cuh", "ibm_internal.cuh"],
    "spread": ["k_tile.cu", "ibm_internal.cuh"],
    "rhs": ["ibm_flow.cu", "ibm_internal.cuh"],
    "cn_scale": ["ibm_flow.cu", "ibm_internal.cuh"],
    "add": ["ibm_flow.cu", "ibm_internal.cuh"],
    "cn_solve": ["ibm_flow.cu", "ibm_internal.cuh"],
    "div": ["ibm_flow.cu", "ibm_internal.cuh"],
    "poisson_scale": ["ibm_flow.cu", "ibm_internal.cuh"],
    "project": ["ibm_flow.cu", "ibm_internal.cuh"],
}


def _code_only(text: str) -> str:
    """C/C++ source without its comments and with runs of white space
    collapsed (string literals kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_digest(key: str) -> str:
    """Digest of the code and flags one profiled kernel is built from:
    comments and layout do not count, and neither does where the repository
    lives (the include path is left out of the flags)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[key] + ["../../include/ibm.h"]:
        p = os.path.normpath(os.path.join(CSRC, name))
        h.update(name.encode())
        with open(p, encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    flags = [f for i, f in enumerate(FLAGS) if f != "-I" and (i == 0 or FLAGS[i - 1] != "-I")]
    h.update(" ".join(ARCH + flags).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of the library."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp.txt")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-L", cuda_lib,
           "-lcufft", "-Xlinker", "-rpath," + cuda_lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
