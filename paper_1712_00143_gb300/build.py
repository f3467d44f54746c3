"""Build libstag.so in-tree with nvcc for sm_103a (GB300).

Each .cu translation unit compiles in its own nvcc process (in parallel);
the objects link into ``paper_1712_00143_gb300/libstag.so``.  Objects are
rebuilt only when a source or header is newer than them.  ``--debug-bounds``
(or build(debug_bounds=True)) builds the bounds-checked
``libstag_debug.so`` from the same sources with -DSTAG_DEBUG_BOUNDS.
"""

import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstag.so")
# the bounds-checked build (every global index checked, violations recorded)
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libstag_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3",
    "-lineinfo",
    "-std=c++17",
    "-Xcompiler",
    "-fPIC",
    "-Xcompiler",
    "-O2",
    "--expt-relaxed-constexpr",
    "-I" + INCLUDE,
    "-I" + CSRC,
]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _compile(src, extra, verbose, build_dir):
    obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
    newest_dep = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep and not extra:
        return obj, ""
    flags = list(extra)
    if build_dir == BUILD_DEBUG:
        flags.append("-DSTAG_DEBUG_BOUNDS")
    cmd = [_nvcc()] + NVCC_FLAGS + flags + ["-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    return obj, (p.stdout + p.stderr) if verbose else ""


def _stamp_ok(build_dir):
    """Objects and library were built on this machine type (x86_64 / aarch64)."""
    stamp = os.path.join(build_dir, "MACHINE")
    try:
        return open(stamp).read().strip() == platform.machine()
    except OSError:
        return False


def build(verbose=False, extra_flags=(), jobs=None, debug_bounds=False):
    """Compile every kernel source and link libstag.so (debug_bounds: the
    bounds-checked libstag_debug.so); returns the library path."""
    build_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug_bounds else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    if not _stamp_ok(build_dir):
        for f in os.listdir(build_dir):
            os.remove(os.path.join(build_dir, f))
        if os.path.exists(lib):
            os.remove(lib)
        with open(os.path.join(build_dir, "MACHINE"), "w") as fh:
            fh.write(platform.machine())
    srcs = _sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, extra_flags, verbose, build_dir), srcs))
    objs = [o for o, _ in results]
    for _, log in results:
        if log:
            sys.stderr.write(log)
    if os.path.exists(lib) and not extra_flags:
        if os.path.getmtime(lib) >= max(os.path.getmtime(o) for o in objs):
            return lib
    tmp = lib + ".tmp"
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else (),
                debug_bounds="--debug-bounds" in sys.argv))
