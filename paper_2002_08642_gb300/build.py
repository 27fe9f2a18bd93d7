"""Build libps.so (the CUDA library behind include/ps.h) in-tree with nvcc.

Translation units are compiled in parallel, one -gencode for sm_103a, then
linked into ``paper_2002_08642_gb300/_build/libps.so``. A rebuild happens
only when a source or header is newer than the library.

``libps_bench.so`` (same folder) holds measurement tooling that bench.py
uses (the device's FMA rate); it is not part of the solver's ABI.
"""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libps.so")
BENCH_LIB = os.path.join(OUT_DIR, "libps_bench.so")
SOURCES = ["ps_api.cu", "ps_f32_a.cu", "ps_f32_b.cu", "ps_f64_a.cu", "ps_f64_b.cu", "ps_noalloc.cu", "ps_massspring.cu"]
BENCH_SOURCES = ["bench_fma_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date():
    if not os.path.exists(LIB) or not os.path.exists(BENCH_LIB):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(BENCH_LIB))
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force=False, verbose=False, extra_flags=()):
    """Compile and link libps.so; returns its path. Raises on compiler errors."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr[-8000:]))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES) + len(BENCH_SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES + BENCH_SOURCES))

    def link(out, parts):
        tmp = out + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *parts, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr[-8000:]))
        os.replace(tmp, out)

    link(LIB, objs[:len(SOURCES)])
    link(BENCH_LIB, objs[len(SOURCES):])
    return LIB

if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
