"""Build libfmgp.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled in parallel with nvcc and the
objects are linked into paper_2205_10879_gb300/libfmgp.so.  Rebuilds only
when a source or header is newer than the library."""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
TARGET = os.path.join(HERE, "libfmgp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def needs_build():
    if not os.path.exists(TARGET):
        return True
    t = os.path.getmtime(TARGET)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(src, verbose):
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [_nvcc()] + ARCH + NVCC_FLAGS + ["-I", INCLUDE, "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    return obj, p.returncode, p.stdout + p.stderr


def build(force=False, verbose=False):
    if not force and not needs_build():
        return TARGET
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), srcs))
    failed = [(o, out) for o, rc, out in results if rc != 0]
    for o, rc, out in results:
        if out.strip() and (verbose or rc != 0 or "warning" in out.lower()):
            sys.stderr.write(out)
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(o) for o, _ in failed))
    tmp = TARGET + f".tmp{os.getpid()}"
    link = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _, _ in results] + ["-lcudart"]
    subprocess.run(link, check=True)
    os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
