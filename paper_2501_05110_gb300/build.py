"""Build the CUDA library (libsapgpu.so) in-tree for sm_103a with nvcc.

Translation units are compiled in parallel and linked with the CUDA runtime.  The output goes to
``paper_2501_05110_gb300/_lib/``; nothing is installed into site-packages.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libsapgpu.so")
SOURCES = ["operator.cu", "apply_rows.cu", "uniform.cu", "adjoint_fields.cu", "probe.cu", "setup.cpp", "sh_tables.cpp"]
# l_max values the uniform-coefficient kernel is compiled for (patterns generated by gen_uniform)
UNIFORM_LMAX = [1, 2, 3, 4, 5]
PATTERNS = os.path.join(OUT, "uniform_patterns.inc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return exe


def _compile(src: str) -> str:
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [_nvcc(), *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-I", OUT,
           "-x", "cu" if src.endswith(".cu") else "c++", "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ["--expt-relaxed-constexpr"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _generate_patterns() -> None:
    """Compile and run the host generator of the uniform kernel's sparsity patterns."""
    exe = os.path.join(OUT, "gen_uniform")
    cmd = [_nvcc(), "-O2", "-std=c++17", "-x", "c++", os.path.join(CSRC, "gen_uniform.cpp"),
           os.path.join(CSRC, "sh_tables.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gen_uniform build failed:\n{r.stdout}\n{r.stderr}")
    r = subprocess.run([exe, PATTERNS + ".tmp", *map(str, UNIFORM_LMAX)], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gen_uniform failed:\n{r.stdout}\n{r.stderr}")
    os.replace(PATTERNS + ".tmp", PATTERNS)


def build(force: bool = False) -> str:
    """Compile and link; returns the path of the shared library."""
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))] + \
        [os.path.join(CSRC, "gen_uniform.cpp")] + \
        [os.path.join(HERE, "..", "include", "sap.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    _generate_patterns()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", LIB + ".tmp", *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
