"""Build libusp.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel, then one shared-object link.
The library lands next to this file; the Python binding loads it from there.
"""

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
LIB = os.path.join(HERE, "libusp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
CUDA_FLAGS = ARCH + ["-lineinfo", "--expt-relaxed-constexpr"] + COMMON
SOURCES = [
    "pencil_kernels.cu",
    "fused3d_kernels.cu",
    "usp_api.cpp",
    "canon.cpp",
    "noalloc.cu",
    "tma_kernels.cu",
    "fno_kernels.cu",
    "fno_api.cpp",
    "block_kernels.cu",
    "variant_api.cpp",
    "tc_kernels.cu",
    "onchip_kernels.cu",
    "split3d_kernels.cu",
    "df_kernels.cu",
    "df_part_small.cu",
    "df_part_p128.cu",
    "df_part_p256.cu",
    "df_part_p384.cu",
    "df_part_p512.cu",
]


def nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _compile(src, extra):
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    if src.endswith(".cu"):
        cmd = [nvcc(), "-c", path, "-o", obj] + CUDA_FLAGS + extra
    else:
        cmd = [nvcc(), "-x", "c++", "-c", path, "-o", obj] + COMMON + extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, r.stderr


def sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(INCLUDE, "usp.h"))
    deps.append(os.path.abspath(__file__))
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force=False, verbose=False, extra=None):
    """Compile every translation unit and link libusp.so.  Returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
