"""Build the irkmg shared library in-tree (sm_103a only).

Each translation unit is compiled by nvcc in parallel and linked into
paper_2202_07381_gb300/_build/libirkmg.so with the static CUDA runtime.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libirkmg.so")
SOURCES = ["host_mesh.cpp", "host_assemble.cpp", "k_patch.cu", "k_linalg.cu", "k_coarse.cu",
           "k_adjoint.cu", "k_patch_big.cu", "k_patch_kron.cu", "k_patch_fixed.cu", "k_ns.cu", "host_kron.cpp", "host_eig.cpp",
           "k_batch.cu", "k_op_fixed.cu", "api.cu", "probe_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the irkmg CUDA library cannot be built")
    return exe


def _compile(src):
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3",
           "-x", "cu", *ARCH, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, ptxas_info=False):
    """Compile every source and link the library; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    global ARCH
    if ptxas_info:
        ARCH = ARCH + ["-Xptxas", "-v"]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err)
    objs = [o for o, _ in results]
    cmd = [_nvcc(), "-shared", *ARCH, "-o", LIB, *objs, "-cudart", "static", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
