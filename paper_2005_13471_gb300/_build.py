"""Build libbsct.so (the CUDA kernels and the C ABI) in-tree for sm_103a with nvcc.

Translation units are compiled in parallel; the FFT convolution source is compiled
once per supported image size.  No cmake, no torch extension machinery.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbsct.so")
FFT_SIZES = (16, 32, 64, 128, 256, 384, 512, 768, 1024, 2048)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbsct")


def _units():
    units = []
    for name in sorted(os.listdir(CSRC)):
        if not name.endswith(".cu"):
            continue
        src = os.path.join(CSRC, name)
        if name == "gram_fft.cu":
            for n in FFT_SIZES:
                units.append((src, os.path.join(BUILD, f"gram_fft_{n}.o"), [f"-DBSCT_FFT_N={n}"]))
        else:
            units.append((src, os.path.join(BUILD, name[:-3] + ".o"), []))
    return units


def _deps_mtime():
    m = 0.0
    for d in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for name in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, name)))
    return m


def _compile(unit):
    src, obj, extra = unit
    cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-I", CSRC, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)} {extra}:\n{r.stderr}")
    return obj


def build(force=False, jobs=None, verbose=False):
    """Compile every .cu under csrc/ and link paper_2005_13471_gb300/libbsct.so."""
    os.makedirs(BUILD, exist_ok=True)
    units = _units()
    newest_src = _deps_mtime()
    todo = [u for u in units if force or not os.path.exists(u[1]) or os.path.getmtime(u[1]) < newest_src]
    jobs = jobs or max(1, min(len(todo) or 1, os.cpu_count() or 4))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            for obj in ex.map(_compile, todo):
                if verbose:
                    print("built", os.path.relpath(obj, HERE), file=sys.stderr)
    objs = [u[1] for u in units]
    if force or todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
