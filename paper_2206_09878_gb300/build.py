"""Build liblmvd.so (and its index-checked variant liblmvd_check.so) in-tree for sm_103a (GB300) with nvcc:
one object per source and variant, compiled in parallel."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblmvd.so")
LIB_CHECK = os.path.join(HERE, "liblmvd_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "fft.cu", "ykernels.cu", "pointwise.cu", "adjoint.cu", "probe.cu", "basis.cpp"]


def _nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblmvd")
    return path


def _compile(src, verbose, checked=False):
    obj = os.path.join(BUILD, src + (".check.o" if checked else ".o"))
    cmd = [_nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-c", os.path.join(CSRC, src), "-o", obj]
    if checked:
        cmd.insert(1, "-DLMVD_CHECK")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def _link(objs, lib):
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)


def build(verbose=False, checked=True):
    """Compile every source of csrc/ and link liblmvd.so next to this file; with checked, also the
    index-checked variant liblmvd_check.so (-DLMVD_CHECK, a testing aid). Returns the path of liblmvd.so."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = [(s, False) for s in SOURCES] + ([(s, True) for s in SOURCES] if checked else [])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(lambda j: _compile(j[0], verbose, j[1]), jobs))
    if verbose:
        for (_, log) in results:
            sys.stderr.write(log)
    objs = [o for (o, _), (_, chk) in zip(results, jobs) if not chk]
    _link(objs, LIB)
    if checked:
        _link([o for (o, _), (_, chk) in zip(results, jobs) if chk], LIB_CHECK)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
