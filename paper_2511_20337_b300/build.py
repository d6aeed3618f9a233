"""Builds libmhd.so (the C-ABI library) in-tree for sm_103a.

    python -m paper_2511_20337_b300.build [--force] [--verbose]

nvcc cross-compiles without a GPU.  The library links the CUDA runtime
statically, so loading it needs no CUDA toolkit on the library path.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
SO = os.path.join(HERE, "libmhd.so")
SOURCES = ["mhd_api.cu", "mhd_batch.cu", "mhd_adjoint.cu", "mhd_domain.cu", "mhd_coop.cu", "mhd_guard.cu"]
DEPS = ["mhd_math.cuh", "mhd_kernels.cuh", "mhd_host.cuh", "mhd_ctx.cuh", "mhd_dual.cuh", "mhd_adjoint.cuh", "mhd_riemann_adj.cuh", "mhd_glm.cuh", "mhd_coop.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if p and (os.path.isabs(p) and os.path.exists(p) or not os.path.isabs(p)):
            return p
    return "nvcc"


def needs_build():
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    files = [os.path.join(CSRC, f) for f in SOURCES + DEPS] + [os.path.join(INCLUDE, h) for h in ("mhd.h", "mhd_probe.h")]
    return any(os.path.getmtime(f) > t for f in files)


def build(force=False, verbose=False):
    """Compile each source to an object in parallel, then link the shared library."""
    if not force and not needs_build():
        return SO
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC", "-I", INCLUDE,
             "-I", CSRC]
    if verbose:
        flags += ["-Xptxas", "-v"]
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    procs = [subprocess.Popen([nvcc(), *flags, "-c", os.path.join(CSRC, s), "-o", o], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for s, o in zip(SOURCES, objs)]
    failed = False
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            failed = True
            sys.stderr.write(out + err)
        elif verbose:
            sys.stderr.write(err)
    if failed:
        raise RuntimeError("nvcc failed building libmhd.so")
    res = subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "static", *objs, "-o", SO + ".tmp"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed linking libmhd.so")
    os.replace(SO + ".tmp", SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
