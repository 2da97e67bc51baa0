"""Build libpt.so in-tree for sm_103a: nvcc for the kernels, g++ for the host layer, compiled in
parallel and linked with nvcc.  No cmake; one -gencode; a few translation units so that a fresh
machine builds in well under a minute."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libpt.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
_lock = threading.Lock()


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _inputs():
    return sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__])


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of libpt.so."""
    with _lock:
        if not force and not _stale():
            return LIB
        cuda = _cuda_home()
        nvcc = os.path.join(cuda, "bin", "nvcc")
        os.makedirs(BUILD, exist_ok=True)
        os.makedirs(LIB_DIR, exist_ok=True)
        inc = ["-I" + INCLUDE, "-I" + CSRC]
        jobs = []
        objs = []
        for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
            obj = os.path.join(BUILD, os.path.basename(src) + ".o")
            objs.append(obj)
            # -fmad=false: every product and sum is rounded on its own, so the megakernel, the
            # wavefront stages and the adjoint compute bit-identical values (ptxas may otherwise fuse
            # a mul and an add into an FMA differently in each kernel, depending on register pressure)
            jobs.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
                         "-Xptxas", "-warn-spills", *inc, "-c", src, "-o", obj])
        for src in sorted(glob.glob(os.path.join(CSRC, "*.cpp"))):
            obj = os.path.join(BUILD, os.path.basename(src) + ".o")
            objs.append(obj)
            jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-pthread", "-Wall", "-I" + os.path.join(cuda, "include"),
                         *inc, "-c", src, "-o", obj])
        procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
        errors = []
        for j, p in zip(jobs, procs):
            out, _ = p.communicate()
            text = out.decode(errors="replace")
            if p.returncode != 0:
                errors.append(" ".join(j) + "\n" + text)
            elif verbose and text.strip():
                print(text)
        if errors:
            raise RuntimeError("libpt build failed:\n" + "\n".join(errors))
        tmp = LIB + f".tmp{os.getpid()}"
        link = [nvcc, ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp, "-lpthread"]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("libpt link failed:\n" + " ".join(link) + "\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
