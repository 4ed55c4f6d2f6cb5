"""Builds libcem.so (the CUDA C-ABI library) in-tree for sm_103a.

Translation units are compiled in parallel with nvcc; the FP64 step, the
tracking kernel and the energy kernels use -fmad=false so that their FP64
arithmetic keeps one fixed IEEE operation order; host code uses
-ffp-contract=off for the same reason.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcem.so")
ROOT = os.path.dirname(HERE)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra flags)
UNITS = [
    ("step_fp64.cu", ["-fmad=false"]),
    ("track.cu", ["-fmad=false"]),
    ("energy.cu", ["-fmad=false"]),
    ("step_fp32.cu", []),
    ("eval_fp32.cu", ["-fmad=false"]),
    ("state_energy_noalloc.cu", ["-fmad=false"]),
    ("surrogate.cu", []),
    ("fragments.cu", []),
    ("tri.cu", ["-fmad=false"]),
    ("api.cpp", []),
]
HEADERS = ["cem_internal.h", "q4_fp64.cuh", "eval_common.cuh", "tri_internal.h"]


def _stale(obj, deps):
    return not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(d) for d in deps)


def _compile(src, extra):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + \
        [os.path.join(ROOT, "include", "cem.h"), os.path.join(ROOT, "include", "cem_surrogate.h")]
    if not _stale(obj, deps):
        return obj
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
           "-I", os.path.join(ROOT, "include"), *extra, "-c", os.path.join(CSRC, src),
           "-o", obj + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libcem.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force:
        for f in os.listdir(OUT_DIR):
            os.remove(os.path.join(OUT_DIR, f))
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(*u), UNITS))
    if _stale(LIB, objs):
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *objs,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
