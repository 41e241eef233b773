"""Build libridfa.so in-tree for sm_103a (nvcc for the device code, g++ for the host compiler).

Run ``python paper_2412_14975_gb300/build_lib.py`` (by path: importing the package needs the
library) or call ``build()``.  The two translation
units compile in parallel; the result is ``paper_2412_14975_gb300/libridfa.so``.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libridfa.so")
BUILD = os.path.join(ROOT, "_build")
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), nvcc


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".h"))] + [os.path.join(INC, "ridfa.h")]


def up_to_date():
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False, extra_nvcc=()):
    if not force and up_to_date():
        return OUT
    cuda, nvcc = _cuda_home()
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    objs = []
    for f in sorted(os.listdir(CSRC)):
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        if f.endswith(".cu"):
            cmd = [nvcc, *GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", INC, "-I", CSRC, *extra_nvcc, "-c", src, "-o", obj]
        elif f.endswith(".cpp"):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INC, "-I", CSRC,
                   "-I", os.path.join(cuda, "include"), "-c", src, "-o", obj]
        else:
            continue
        objs.append(obj)
        if verbose:
            print(" ".join(cmd), flush=True)
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in jobs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("libridfa build failed:\n" + msg)
    tmp = OUT + f".tmp{os.getpid()}"
    link = [nvcc, *GENCODE, "-shared", "-cudart", "shared", "-o", tmp, *objs,
            "-Xlinker", "-rpath=" + os.path.join(cuda, "lib64")]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.check_call(link)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
