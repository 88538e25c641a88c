"""Build the CUDA library libfcsdnn.so in-tree for sm_103a (nvcc + g++)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libfcsdnn.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(verbose=False, extra=()):
    """Compile csrc/*.cu and csrc/*.cpp into _lib/libfcsdnn.so; returns the path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    obj_cu = os.path.join(OUT_DIR, "fcs_api.o")
    obj_cpp = os.path.join(OUT_DIR, "fcs_tables.o")
    host_flags = "-fPIC,-O2,-ffp-contract=off"
    cmds = [
        [nvcc, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", host_flags,
         "-Xptxas", "-v" if verbose else "-O3", *extra, "-o", obj_cu, os.path.join(SRC, "fcs_api.cu")],
        ["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-o", obj_cpp,
         os.path.join(SRC, "fcs_tables.cpp")],
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out)
        if p.returncode != 0:
            raise RuntimeError("build failed: " + " ".join(c))
    link = [nvcc, "-shared", *ARCH, "-o", LIB, obj_cu, obj_cpp]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        sys.stdout.write(r.stdout)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
