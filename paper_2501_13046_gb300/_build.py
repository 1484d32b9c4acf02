"""Build the CUDA library libctt_mg.so in-tree with nvcc for sm_103a.

The translation units compile in parallel; the result sits next to this file
and is what the ctypes binding loads.  No torch extension machinery is used:
the library is a plain C-ABI shared object.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libctt_mg.so")
OBJDIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
# one engine unit per (precision, order, boundary variant): they compile in parallel
ENGINE = ["mg_engine_f32_o2_periodic.cu", "mg_engine_f32_o2_robin.cu", "mg_engine_f32_o2_sym.cu", "mg_engine_f32_o4_periodic.cu", "mg_engine_f32_o4_robin.cu", "mg_engine_f32_o4_sym.cu", "mg_engine_f64_o2_periodic.cu", "mg_engine_f64_o2_robin.cu", "mg_engine_f64_o2_sym.cu", "mg_engine_f64_o4_periodic.cu", "mg_engine_f64_o4_robin.cu", "mg_engine_f64_o4_sym.cu"]
SOURCES = ["ctt_mg.cu", *ENGINE, "mg_noalloc.cu", "mg_warmstart.cu", "unet_conv.cu", "unet_glue.cu"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def deps():
    out = [os.path.join(HERE, "..", "include", f) for f in ("ctt_mg.h", "ctt_unet.h")]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def build(force=False, verbose=False, extra=()):
    if not force and not _stale(LIB, deps()):
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ())
