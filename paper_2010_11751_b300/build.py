"""Build liblbm.so (the CUDA library) in-tree for sm_103a.

Every translation unit under csrc/ is compiled by nvcc in parallel into
_build/, then linked into paper_2010_11751_b300/liblbm.so with the CUDA runtime
linked statically.  A rebuild happens when any source or header is newer than
the library.

build(debug=True) makes liblbm_debug.so instead: the same sources compiled
with -DLBM_DEBUG into _build/debug/, whose kernels check every population,
cell, flag and staged-copy index against the arrays' extents and record the
first fault per handle instead of touching memory out of bounds
(lbm_debug_check reads it).  It holds three collision models (BGK-W2, TRT and
the cumulant model), which keeps its build short.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "liblbm.so")
LIB_DEBUG = os.path.join(PKG, "liblbm_debug.so")
BUILD_DEBUG = os.path.join(BUILD, "debug")
# the model translation units of the bounds-checked build
DEBUG_MODELS = ("model_bgk_w2.cu", "model_trt.cu", "model_k.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def _sources(debug=False):
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if debug:
        srcs = [s for s in srcs if not os.path.basename(s).startswith("model_")
                or os.path.basename(s) in DEBUG_MODELS]
    return srcs


def _inputs():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date(debug=False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(src, extra, force=False, objdir=BUILD, reuse=True):
    obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
    if not force and reuse and os.path.exists(obj):
        t = os.path.getmtime(obj)
        if all(os.path.getmtime(p) <= t for p in [src, os.path.abspath(__file__)] + _headers()):
            return obj, ""
    cmd = [_nvcc()] + FLAGS + ARCH + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj, r.stderr


HEAVY = ("model_rr.cu", "model_bgk_w2.cu", "model_trt.cu", "model_k.cu", "model_cm.cu", "model_chm.cu")



def _heaviest_first(item):
    name = os.path.basename(item[0])
    return (name not in HEAVY, HEAVY.index(name) if name in HEAVY else 0, item[2], name)


def build_all(force: bool = False, jobs: int | None = None) -> tuple[str, str]:
    """liblbm.so and liblbm_debug.so, their translation units compiled in one pool (heaviest
    first), so that the two builds share the cores."""
    todo = []
    for debug in (False, True):
        if force or not up_to_date(debug):
            objdir = BUILD_DEBUG if debug else BUILD
            os.makedirs(objdir, exist_ok=True)
            todo += [(src, debug, objdir) for src in _sources(debug)]
    if todo:
        todo.sort(key=_heaviest_first)
        jobs = jobs or max(1, os.cpu_count() or 1)
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            list(ex.map(lambda t: _compile(t[0], ["-DLBM_DEBUG"] if t[1] else [], force, t[2], reuse=True), todo))
        for debug in sorted({t[1] for t in todo}):
            objdir = BUILD_DEBUG if debug else BUILD
            lib = LIB_DEBUG if debug else LIB
            objs = [os.path.join(objdir, os.path.basename(src)[:-3] + ".o") for src in _sources(debug)]
            tmp = lib + ".tmp"
            subprocess.run([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
            os.replace(tmp, lib)
    return LIB, LIB_DEBUG


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, extra=(), debug=False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(debug):
        return lib
    objdir = BUILD_DEBUG if debug else BUILD
    os.makedirs(objdir, exist_ok=True)
    srcs = _sources(debug)
    # heaviest units first so the parallel build finishes sooner (the FP64 BGK-W2 and TRT
    # kernels come in two ranges of their fast path)
    srcs.sort(key=lambda s: _heaviest_first((s, debug, "")))
    jobs = jobs or max(1, os.cpu_count() or 1)
    flags = list(extra) + (["-DLBM_DEBUG"] if debug else [])
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        # objects are reused only by builds without extra nvcc flags
        results = list(ex.map(lambda s: _compile(s, flags, force, objdir, reuse=not extra), srcs))
    if verbose:
        for _, err in results:
            if err:
                print(err, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    subprocess.run([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    t = build(force="--force" in sys.argv, verbose="-v" in sys.argv,
              extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], debug="--debug" in sys.argv)
    print(t)
