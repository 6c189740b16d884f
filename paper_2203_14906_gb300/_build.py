"""Build the in-tree CUDA library ``_lib/libpa_hodmas.so`` for sm_103a.

Each translation unit is compiled by its own ``nvcc -c`` process (the
fused-kernel instantiations are split by order so they compile in
parallel), then linked with ``nvcc -shared``.  The CUDA runtime is linked
statically.  ``checked=True`` builds a variant with device-side bounds
checks (``PA_CHECK_BOUNDS``) that record an error word instead of
accessing memory out of range.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "_lib")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def lib_path(checked: bool = False) -> str:
    return os.path.join(LIBDIR, "libpa_hodmas_checked.so" if checked else "libpa_hodmas.so")


def _nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the beamformer")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(checked: bool = False, force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of the shared library."""
    target = lib_path(checked)
    with _lock:
        if not force and not _stale(target):
            return target
        nvcc = _nvcc()
        tag = "checked" if checked else "release"
        objdir = os.path.join(LIBDIR, "obj_" + tag)
        os.makedirs(objdir, exist_ok=True)
        flags = ARCH + [
            "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-Xptxas", "-v", "-I", INCLUDE, "-I", CSRC,
        ]
        if checked:
            flags.append("-DPA_CHECK_BOUNDS=1")

        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc] + flags + ["-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-6000:]}")
            return obj, r.stderr

        srcs = _sources()
        with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(compile_one, srcs))
        with open(os.path.join(LIBDIR, f"ptxas_{tag}.log"), "w") as f:
            for (obj, err) in results:
                f.write(f"== {os.path.basename(obj)}\n{err}\n")
        tmp = target + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, target)
        if verbose:
            print(f"built {target}")
        return target


if __name__ == "__main__":
    import sys

    print(build(checked="--checked" in sys.argv, force="--force" in sys.argv, verbose=True))
