"""Build libssj.so in-tree with nvcc for sm_103a (GB300), and its checked
twin libssj_checked.so (-DSSJ_CHECKED: every index of the plan and verify
kernels is tested against its array's extent; a bad one sets an error bit
instead of faulting), which tests load with SSJ_LIBRARY=checked.

Each translation unit is compiled to an object in parallel, then linked
into one shared library next to this file.  A stamp of the sources and
flags skips the rebuild when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libssj.so")
LIB_CHECKED = os.path.join(HERE, "libssj_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "--expt-relaxed-constexpr", "-I", INCLUDE]
SOURCES = ["api.cu", "verify.cu", "layout.cu", "noalloc.cu", "probe.cu", "candgen.cu", "feeder.cpp", "groups.cpp", "renumber.cpp", "serve_driver.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stamp(extra: list[str]) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    for name in sorted(os.listdir(INCLUDE)):
        with open(os.path.join(INCLUDE, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + extra).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Both libraries (the checked one in parallel with the product one); returns libssj.so's path."""
    extra = list(extra_flags or [])
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        checked = ex.submit(_build_one, LIB_CHECKED, os.path.join(BUILD, "checked"), force, verbose,
                            extra + ["-DSSJ_CHECKED"])
        lib = _build_one(LIB, BUILD, force, verbose, extra)
        checked.result()
    return lib


def _build_one(lib_path: str, build_dir: str, force: bool, verbose: bool, extra: list[str]) -> str:
    os.makedirs(build_dir, exist_ok=True)
    stamp = _stamp(extra)
    stamp_file = os.path.join(build_dir, "libssj.stamp")
    if not force and os.path.exists(lib_path) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return lib_path
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, src + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, *NVCC_FLAGS, *extra, "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    res = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
