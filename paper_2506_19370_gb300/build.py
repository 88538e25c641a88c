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
    """Compile csrc/*.cu and csrc/*.cpp (in parallel) into _lib/libfcsdnn.so; returns the path."""
    import glob
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    host_flags = "-fPIC,-O2,-ffp-contract=off"
    cmds, objs = [], []
    for src in sorted(glob.glob(os.path.join(SRC, "*.cu"))):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", host_flags,
                     "-Xptxas", "-v" if verbose else "-O3", *extra, "-o", obj, src])
    for src in sorted(glob.glob(os.path.join(SRC, "*.cpp"))):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-4] + ".o")
        objs.append(obj)
        cmds.append(["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-o", obj, src])
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    failed = None
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed = c
    if failed:
        raise RuntimeError("build failed: " + " ".join(failed))
    link = [nvcc, "-shared", *ARCH, "-o", LIB, *objs]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        sys.stdout.write(r.stdout)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
