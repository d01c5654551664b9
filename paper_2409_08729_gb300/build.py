"""Build the CUDA library in-tree for sm_103a (nvcc, no cmake).

Two libraries from the same sources: liblogbessel.so (release) and
liblogbessel_checks.so (LB_CHECKS: every shared-list, queue and pair index
checked against its bound, failures recorded in a status word; see
logbessel_check_status).  Every translation unit compiles in its own nvcc
process, all of them in parallel, then each library is linked."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liblogbessel.so")
CHECKS_LIB_PATH = os.path.join(BUILD_DIR, "liblogbessel_checks.so")

SOURCES = ["logbessel.cu", "lb_peaks.cu", "lb_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(path):
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in _deps())


def build_library(force=False, verbose=False, checks=True):
    """Compile the library (and, with checks, the checked library) if any
    source is newer; return the release library's path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    variants = [(LIB_PATH, [])]
    if checks:
        variants.append((CHECKS_LIB_PATH, ["-DLB_CHECKS"]))
    variants = [(lib, defs) for lib, defs in variants if force or _stale(lib)]
    if not variants:
        return LIB_PATH
    tag = "%d" % os.getpid()
    jobs = []
    for lib, defs in variants:
        objs = []
        for src in SOURCES:
            obj = os.path.join(BUILD_DIR, "%s.%s%s.o" % (src[:-3], "checks." if defs else "", tag))
            cmd = [nvcc()] + ARCH + FLAGS + defs + ["-I" + INCLUDE, "-I" + CSRC, "-c", os.path.join(CSRC, src),
                                                      "-o", obj]
            if verbose:
                print(" ".join(cmd))
            jobs.append(subprocess.Popen(cmd))
            objs.append(obj)
        variants_objs = (lib, objs)
        jobs.append(variants_objs)
    procs = [j for j in jobs if isinstance(j, subprocess.Popen)]
    failed = [p for p in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(failed[0].returncode, failed[0].args)
    for lib, objs in (j for j in jobs if isinstance(j, tuple)):
        tmp = lib + ".tmp" + tag
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, lib)
        for o in objs:
            os.remove(o)
    return LIB_PATH


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
