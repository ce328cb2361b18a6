"""Build libugkwp.so (the C-ABI library) in-tree for sm_103a.

Kernels that feed the particle path (k_cells.cu, k_particles.cu) are compiled
with --fmad=false so that their arithmetic is one IEEE operation per written
operation; the wave-flux kernel keeps fused multiply-adds.  Host C++ is built
with -ffp-contract=off for the same reason (it computes the tracking planes).
The CUDA runtime is linked statically so the library loads without a driver
(only its compute calls need a GPU).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libugkwp.so")
ROOT = os.path.dirname(PKG)
INC = os.path.join(ROOT, "include")

GENCODE = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_COMMON = ["-O3", "-lineinfo", "-std=c++17", GENCODE, "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
               f"-I{INC}", "--expt-relaxed-constexpr"]
CU_UNITS = {
    "k_cells.cu": ["--fmad=false"],
    "k_particles.cu": ["--fmad=false"],
    "k_flux.cu": [],
    "k_noalloc.cu": ["--fmad=false"],
    "k_adjoint.cu": [],
}
CPP_UNITS = ["api.cpp", "mesh.cpp"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(SRC, f) for f in list(CU_UNITS) + CPP_UNITS] + \
        [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".hpp", ".h"))] + \
        [os.path.join(INC, "ugkwp.h"), os.path.abspath(__file__)]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT, exist_ok=True)
    jobs = []
    for f, extra in CU_UNITS.items():
        obj = os.path.join(OUT, f + ".o")
        jobs.append([nvcc, *NVCC_COMMON, *extra, "-c", os.path.join(SRC, f), "-o", obj])
    for f in CPP_UNITS:
        obj = os.path.join(OUT, f + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", f"-I{INC}",
                     f"-I{os.path.join(cuda, 'include')}", "-c", os.path.join(SRC, f), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        for log in logs:
            if log.strip():
                print(log)
    objs = [os.path.join(OUT, f + ".o") for f in list(CU_UNITS) + CPP_UNITS]
    tmp = LIB + ".tmp"
    run([nvcc, "-shared", GENCODE, "-cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
