"""Build libk2svd.so and libk2probe.so in-tree with nvcc for sm_103a.

Each .cu file under csrc/ is compiled in parallel into csrc/_build/*.o.  The method's
sources are linked into csrc/libk2svd.so (include/k2svd.h); the measurement probes
(k2_probe.cu, include/k2probe.h) into a library of their own, csrc/libk2probe.so, so the
product library holds no measurement code.  The numerics flags keep IEEE semantics: no
flush to zero, correctly rounded division and square root, and no contraction of a*b+c
into an fma (the paper's formulas call fma explicitly where they want one).
"""
import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(CSRC, "_build")
LIB = os.path.join(CSRC, "libk2svd.so")
PROBE_LIB = os.path.join(CSRC, "libk2probe.so")
PROBE_SRC = "k2_probe.cu"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NUMERICS = ["-ftz=false", "-prec-div=true", "-prec-sqrt=true", "--fmad=false"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _deps():
    return glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale():
    if not os.path.exists(LIB) or not os.path.exists(PROBE_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB))
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force=False, verbose=False):
    """Compile every CUDA source and link libk2svd.so and libk2probe.so; returns the
    path of libk2svd.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cc = nvcc()

    def one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc] + ARCH + FLAGS + NUMERICS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(one, srcs))
    probe = [o for o, s in zip(objs, srcs) if os.path.basename(s) == PROBE_SRC]
    method = [o for o, s in zip(objs, srcs) if os.path.basename(s) != PROBE_SRC]
    for out, parts in ((LIB, method), (PROBE_LIB, probe)):
        tmp = out + ".tmp.%d" % os.getpid()
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + parts + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(tmp, out)
    return LIB

if __name__ == "__main__":
    print(build(force=True, verbose=True))
