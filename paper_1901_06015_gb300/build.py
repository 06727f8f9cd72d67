"""Build the CUDA library ``libmxgemm.so`` in-tree for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then linked
into one shared library with a plain C ABI (``include/mxgemm.h``). Rebuilds only
when a source or header is newer than the library.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmxgemm.so")
# Debug build: the same library compiled with -DMXG_DEBUG_BOUNDS, whose pack kernels and
# epilogues check every element address against the extent their arguments describe and
# report a violation in the device error word (mxg_check_device_error) instead of
# accessing it. Built on request only (build(debug_bounds=True)).
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libmxgemm_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(CSRC, "exports.map")] + \
        [os.path.join(ROOT, "include", "mxgemm.h"), os.path.abspath(__file__)]


def up_to_date(debug_bounds=False):
    lib = LIB_DEBUG if debug_bounds else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force=False, verbose=False, debug_bounds=False):
    lib_path = LIB_DEBUG if debug_bounds else LIB
    build_dir = BUILD_DEBUG if debug_bounds else BUILD
    if not force and up_to_date(debug_bounds):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=default",
              "-I", os.path.join(ROOT, "include")] + (["-DMXG_DEBUG_BOUNDS"] if debug_bounds else [])

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc] + ARCH + common + ["-lineinfo", "--expt-relaxed-constexpr", "-c", src, "-o", obj]
        else:
            cmd = [nvcc] + common + ["-x", "cu", "-c", src, "-o", obj] + ARCH
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + \
        ["-Xlinker", "--version-script=" + os.path.join(CSRC, "exports.map")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
