"""Build libpd.so in-tree: nvcc for the CUDA sources (sm_103a only), g++ with
OpenMP for the host setup, one shared library with a C ABI (include/pd.h)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libpd.so")
OBJ = os.path.join(HERE, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["k_local.cu", "k_sparse.cu", "k_dense.cu", "k_mixed.cu", "k_chol_ll.cu", "pd_api.cu", "k_noalloc.cu", "k_tc.cu", "k_mlp.cu",
      "k_detect.cu", "k_setup.cu"]
CPP = ["host_setup.cpp", "pd_host.cpp"]
HEADERS = ["kernels.h", "host_setup.h", "solver.h", "mixed.h", "tc.h", "tc_dev.cuh", "mlp.h", "lowp_tile.cuh", "chol_ll.h",
           "df_arith.cuh", "setup_dev.h"]


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("build step failed: " + os.path.basename(cmd[-1]))


def build(verbose=False):
    os.makedirs(OBJ, exist_ok=True)
    hdrs = [os.path.join(SRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "pd.h")]
    objs = []
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + SRC]
    for f in CU:
        src = os.path.join(SRC, f)
        o = os.path.join(OBJ, f + ".o")
        if _newer(o, [src] + hdrs):
            _run([NVCC] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                  "-Xptxas", "-v" if verbose else "-O3"] + inc + ["-c", src, "-o", o])
        objs.append(o)
    for f in CPP:
        src = os.path.join(SRC, f)
        o = os.path.join(OBJ, f + ".o")
        if _newer(o, [src] + hdrs):
            _run(["g++", "-O3", "-mavx2", "-mfma", "-fopenmp", "-fPIC", "-std=c++17"] + inc + ["-c", src, "-o", o])
        objs.append(o)
    if _newer(OUT, objs):
        _run([NVCC] + ARCH + ["-shared", "-Xcompiler", "-fopenmp", "-o", OUT] + objs + ["-lcudart", "-lgomp"])
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
