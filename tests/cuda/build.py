"""Builds the test-only CUDA helpers (tests/_build/*.so)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "_build")


def build():
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(HERE, "curand_philox_ref.cu")
    lib = os.path.join(OUT, "libcurand_philox_ref.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                        "-Xcompiler", "-fPIC", "-shared", src, "-o", tmp], check=True)
        os.replace(tmp, lib)
    return lib
