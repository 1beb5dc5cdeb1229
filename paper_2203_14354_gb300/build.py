"""Build the CUDA library (liblxo.so, sm_103a) in-tree under _build/.

nvcc compiles the kernels and the C-ABI layer, g++ the host BVH builder; the
objects are compiled in parallel and linked with the static CUDA runtime so
the library has no dependency beyond the driver."""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblxo.so")
# the checked build: every node / record / cell / tally index compared with its
# array size in the kernels (LXO_CHECK_BOUNDS), for debugging; never the default
LIB_CHECKED = os.path.join(OUT_DIR, "checked", "liblxo.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["lxo_kernels.cu", "lxo_api.cu"]
CXX_SOURCES = ["bvh_build.cpp"]
HEADERS = ["lxo_internal.h", os.path.join("..", "..", "include", "lxo.h")]


def _newest_input():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES + HEADERS] + [__file__]
    return max(os.path.getmtime(f) for f in files)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force=False, verbose=False, checked=False):
    lib = LIB_CHECKED if checked else LIB
    out_dir = os.path.dirname(lib)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cuda_home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    defs = ["-DLXO_CHECK_BOUNDS=1"] if checked else []
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        jobs.append((obj, [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-v", "-Xcompiler", "-fPIC",
                           *defs, "-c", os.path.join(CSRC, src), "-o", obj]))
    for src in CXX_SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        jobs.append((obj, ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", f"-I{cuda_home}/include", "-c",
                           os.path.join(CSRC, src), "-o", obj]))
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        logs = list(ex.map(lambda j: _run(j[1]), jobs))
    with open(os.path.join(out_dir, "ptxas.log"), "w") as f:
        f.write("\n".join(logs))
    tmp = lib + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp] + [j[0] for j in jobs])
    os.replace(tmp, lib)
    if verbose:
        print("\n".join(logs))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
