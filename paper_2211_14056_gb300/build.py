"""Build the CUDA library in-tree for sm_103a (GB300).

    python -m paper_2211_14056_gb300.build [--verbose-ptxas]

Compiles every ``csrc/*.cu`` translation unit in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) and links
``paper_2211_14056_gb300/lib/libmadflow_gb300.so``.  Objects go to
``paper_2211_14056_gb300/_build/``.  Only sources newer than their object are
recompiled.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libmadflow_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe) and shutil.which(exe) is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return exe


def flags(verbose_ptxas=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                "-I", CSRC, "-I", os.path.join(ROOT, "include")]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src, obj, fl):
    cmd = [nvcc(), "-c", src, "-o", obj] + fl
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(verbose_ptxas=False, force=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    fl = flags(verbose_ptxas)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "madflow_gb300.h"))
    newest_header = max(os.path.getmtime(h) for h in headers)
    srcs = sorted(os.path.join(CSRC, s) for s in os.listdir(CSRC) if s.endswith(".cu"))
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    todo = [(s, o) for s, o in zip(srcs, objs)
            if force or verbose_ptxas or not os.path.exists(o)
            or os.path.getmtime(o) < max(os.path.getmtime(s), newest_header)]
    logs = {}
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or len(todo)) as ex:
            futs = {ex.submit(_compile, s, o, fl): s for s, o in todo}
            for f in cf.as_completed(futs):
                logs[os.path.basename(futs[f])] = f.result()
    if todo or not os.path.exists(LIB):
        cmd = [nvcc(), "-shared", "-o", LIB] + objs + ARCH + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB, logs


if __name__ == "__main__":
    lib, logs = build(verbose_ptxas="--verbose-ptxas" in sys.argv, force="--force" in sys.argv)
    for k, v in sorted(logs.items()):
        if v.strip():
            print(f"== {k}\n{v}")
    print(lib)
