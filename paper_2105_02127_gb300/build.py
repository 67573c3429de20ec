"""Build libteno.so in-tree (paper_2105_02127_gb300/_build/) for sm_103a.

Four translation units compiled in parallel -- the CUDA kernels, the
no-allocation CFL entry point and the FMA pipe-peak measurement with nvcc,
the host runtime with g++ (OpenMP) --
linked by nvcc into one shared library with the C ABI of include/teno.h.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libteno.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["teno_kernels.cu", "teno_noalloc.cu", "teno_peaks.cu", "teno_host.cpp"]
HEADERS = [os.path.join(CSRC, "teno_internal.h"), os.path.join(ROOT, "include", "teno.h")]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = "nvcc"
    inc = os.path.join(cuda, "include")
    pid = os.getpid()
    ko = os.path.join(OUT_DIR, f"teno_kernels.{pid}.o")
    no = os.path.join(OUT_DIR, f"teno_noalloc.{pid}.o")
    po = os.path.join(OUT_DIR, f"teno_peaks.{pid}.o")
    ho = os.path.join(OUT_DIR, f"teno_host.{pid}.o")
    cmd_k = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
             "-diag-suppress", "177", "-c", os.path.join(CSRC, "teno_kernels.cu"), "-o", ko]
    cmd_n = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
             "-c", os.path.join(CSRC, "teno_noalloc.cu"), "-o", no]
    cmd_p = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
             "-c", os.path.join(CSRC, "teno_peaks.cu"), "-o", po]
    cmd_h = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-ffp-contract=off",
             "-Wno-maybe-uninitialized", f"-I{inc}", "-c", os.path.join(CSRC, "teno_host.cpp"),
             "-o", ho]
    cmds = (cmd_k, cmd_n, cmd_p, cmd_h)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in cmds]
    for p, c in zip(procs, cmds):
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(c)}\n{out.decode(errors='replace')}")
        if verbose and out:
            print(out.decode(errors="replace"))
    tmp = LIB + f".tmp{pid}"
    cmd_l = [nvcc, *ARCH, "-shared", "-o", tmp, ko, no, po, ho, "-Xcompiler", "-fopenmp"]
    r = subprocess.run(cmd_l, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd_l)}\n{r.stdout.decode(errors='replace')}")
    os.replace(tmp, LIB)
    for f in (ko, no, po, ho):
        try:
            os.remove(f)
        except OSError:
            pass
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
