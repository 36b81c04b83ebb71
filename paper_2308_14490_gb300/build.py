"""Build libaz.so (the CUDA library behind include/az.h) in-tree with nvcc.

Every translation unit is compiled for sm_103a only, in parallel, then linked
into paper_2308_14490_gb300/libaz.so (CUDA runtime linked statically).
Re-running is cheap: objects are rebuilt only when a source or header changed.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libaz.so")
SOURCES = ["kernels.cu", "lowrank.cu", "lowrank_large.cu", "tc_tsgram.cu", "az_api.cu", "profile.cu", "noalloc.cu",
           "dfgemm.cu", "hqr.cu", "cluster_sketch.cu"]
HEADERS = ["az_internal.cuh", "fft.cuh", "fft_reg.cuh", "kernels.cuh", "lowrank.cuh", "lowrank_large.cuh", "profile.cuh",
           "tc_tsgram.cuh", "dfgemm.cuh", "hqr.cuh", "cluster_sketch.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the AZ CUDA library cannot be built")


def _newest_dep():
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "az.h"), __file__]
    return max(os.path.getmtime(d) for d in deps if os.path.exists(d))


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    dep_t = _newest_dep()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), dep_t):
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    if jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        libdir = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
        run([nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-cudart", "static", "-L" + libdir, "-lcublas", "-lcusolver",
             "-Xlinker", "-rpath," + libdir])
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
