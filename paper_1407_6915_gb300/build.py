"""Builds libfftseg.so (the C-ABI library) in-tree for sm_103a with nvcc.

Each translation unit under csrc/ compiles in parallel; objects are cached by
modification time under paper_1407_6915_gb300/_build/.  No torch headers are
involved: the library is plain CUDA C++ behind the C ABI in include/fftseg.h.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfftseg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the fftseg CUDA library cannot be built")


def _deps():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (os.path.basename(src), r.stdout, r.stderr))
    return obj


def build(force: bool = False, verbose: bool = False, extra=None, debug: bool = False) -> str:
    """Builds libfftseg.so, or with debug=True the self-checking variant
    libfftseg_debug.so (-DFFTSEG_DEBUG: kernels check their shared-memory and
    ring indices and report a bad one through fftseg_plan_check)."""
    nvcc = _nvcc()
    build_dir = BUILD + ("_debug" if debug else "")
    lib_path = LIB[:-3] + "_debug.so" if debug else LIB
    if debug:
        extra = list(extra or []) + ["-DFFTSEG_DEBUG"]
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    newest_dep = max([os.path.getmtime(d) for d in _deps()] + [0.0])
    todo, objs = [], []
    for s in srcs:
        o = os.path.join(build_dir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), newest_dep):
            todo.append((s, o))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(_compile, nvcc, s, o, list(extra or [])) for s, o in todo]
            for f in futs:
                f.result()
    if todo or not os.path.exists(lib_path):
        tmp = lib_path + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib_path)
    if verbose:
        print("built", lib_path)
    return lib_path


if __name__ == "__main__":
    build(force=True, verbose=True)
