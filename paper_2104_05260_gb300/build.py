"""Build libhsma.so in-tree (CUDA kernels for sm_103a + host C++).

Each translation unit compiles in parallel; the shared library links the CUDA
runtime statically, so it needs only the driver at run time.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhsma.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU = ["pair.cu", "kernels.cu", "noalloc.cu", "md.cu", "tree.cu"]
CPP = ["geometry.cpp", "api.cpp", "serve.cpp", "md.cpp"]
HEADERS = ["geometry.hpp", "internal.hpp", "api_internal.hpp", "md_internal.hpp"]


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc):
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _commands(extra_cu=()):
    nvcc = _nvcc()
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(_cuda_home(nvcc), "include")]
    cmds = []
    for f in CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        cmds.append((obj, [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "--ftz=true",
                           "-Xcompiler", "-fPIC,-ffp-contract=off", *inc, *extra_cu,
                           "-c", src, "-o", obj]))
    cxx = shutil.which("g++") or "g++"
    for f in CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        cmds.append((obj, [cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", *inc,
                           "-c", src, "-o", obj]))
    link = [nvcc, "-shared", *ARCH, "-o", LIB] + [o for o, _ in cmds] + ["-lpthread", "-ldl", "-lrt"]
    return cmds, link


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, f) for f in CU + CPP + HEADERS]
    srcs += [os.path.join(ROOT, "include", "hsma.h"), __file__]
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force=False, verbose=False, extra_cu=()):
    """Compile libhsma.so if any source changed; return its path."""
    if not force and not extra_cu and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cmds, link = _commands(extra_cu)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        logs = list(ex.map(run, [c for _, c in cmds]))
    logs.append(run(link))
    if verbose:
        print("\n".join(l for l in logs if l.strip()))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra_cu=tuple(sys.argv[1:])))
