"""Build the CUDA library (libviper.so) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by its own nvcc process (in
parallel), then linked into paper_1906_05260_gb300/libviper.so.  Objects go to
paper_1906_05260_gb300/_build/ (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libviper.so")
SOURCES = ["capi.cu", "rod.cu", "contact.cu", "io.cu", "query.cu", "noalloc.cu", "serve.cu", "frame.cu", "batch.cu"]
HEADERS = ["viper_device.cuh", "viper_impl.h", "phases.cuh", os.path.join("..", "..", "include", "viper.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile and link libviper.so if any source is newer than it."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input() and not verbose_ptxas:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static" if False else "-cudart=static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


WAIT_TEST_LIB = os.path.join(HERE, "libviper_waittest.so")


def build_wait_test(force: bool = False) -> str:
    """A test build of the library (libviper_waittest.so) whose frame kernel has
    a short barrier spin limit and leaves the last CTA's barrier arrival out,
    so that every grid-barrier wait runs out: the bounded-wait path (timeout
    error, every CTA returns) exercised without a hang.  The other objects are
    those of libviper.so."""
    build()
    if not force and os.path.exists(WAIT_TEST_LIB) and os.path.getmtime(WAIT_TEST_LIB) >= _newest_input():
        return WAIT_TEST_LIB
    obj = os.path.join(BUILD, "frame_waittest.o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-DVIPER_TEST_MISSING_ARRIVAL", "-DVIPER_BARRIER_SPINS=4096", "-c",
           os.path.join(CSRC, "frame.cu"), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for the wait-test frame.cu:\n{r.stdout}\n{r.stderr}")
    objs = [os.path.join(BUILD, src.replace(".cu", ".o")) for src in SOURCES if src != "frame.cu"] + [obj]
    tmp = WAIT_TEST_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart=static"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, WAIT_TEST_LIB)
    return WAIT_TEST_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
