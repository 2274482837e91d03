"""Compile the hop engine (CUDA for sm_103a + host runtime) into _build/libpsc.so.

The library is built in-tree so the loader below always picks up this build.
Translation units compile in parallel; a rebuild happens only when a source,
header or flag changed.
"""
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpsc.so")
SOURCES = ["psc_kernels.cu", "psc_sort.cu", "psc_api.cpp", "psc_batch.cpp", "psc_tune.cpp", "psc_static.cu", "psc_slab.cpp",
           "psc_readout.cu"]
HEADERS = [os.path.join(CSRC, "psc_internal.h"), os.path.join(CSRC, "psc_runtime.h"), os.path.join(CSRC, "psc_tiles.cuh"), os.path.join(CSRC, "psc_tiles_lean.cuh"), os.path.join(CSRC, "psc_slab.cuh"), os.path.join(CSRC, "psc_subvol.cuh"), os.path.join(CSRC, "psc_readout.h"), os.path.join(ROOT, "include", "psc.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O3",
                "-Xptxas", "-O3", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _nvcc():
    cand = shutil.which("nvcc") or os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the hop engine needs the CUDA toolkit to build")
    return cand


def _digest():
    h = hashlib.sha256()
    for p in [os.path.join(CSRC, s) for s in SOURCES] + HEADERS + [os.path.abspath(__file__)]:
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libpsc.so if needed; return its path."""
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "libpsc.sha256")
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(OUT, src + ".o")
        objs.append(obj)
        cmd = [nvcc] + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed on " + ", ".join(failed))
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
