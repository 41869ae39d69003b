"""Build libsvsim.so in-tree: CUDA sources for sm_103a with nvcc, host C++
with g++, compiled in parallel and linked with nvcc (static cudart).

    python -m paper_2604_12256_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsvsim.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found")


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    return cu, cpp


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INC, "*.h")) + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


# device headers compiled at run time into specialised sweep kernels (jit.cpp)
JIT_HEADERS = ("chunk_dev.cuh", "program.h", "dfloat.h")


def _write_jit_headers() -> str:
    """C++ source holding the run-time compiler's headers as strings."""
    out = os.path.join(BUILD, "jit_headers.cpp")
    lines = ["// generated by build.py from csrc: headers of the specialised sweep kernels",
             "namespace svs {", f"extern const int kJitHeaderCount = {len(JIT_HEADERS)};",
             "extern const char *const kJitHeaderNames[] = {" +
             ", ".join(f'"{h}"' for h in JIT_HEADERS) + "};",
             "extern const char *const kJitHeaderSources[] = {"]
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h)) as f:
            text = f.read()
        assert ")svsjit\"" not in text
        lines.append('R"svsjit(' + text + ')svsjit",')
    lines += ["};", "}  // namespace svs", ""]
    data = "\n".join(lines)
    if not os.path.exists(out) or open(out).read() != data:
        with open(out, "w") as f:
            f.write(data)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp = _sources()
    cpp.append(_write_jit_headers())
    common_inc = ["-I", INC, "-I", CSRC]
    jobs = []
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", "--use_fast_math=false",
               "-Xcompiler", "-fPIC", "-Xptxas", "-O3"] + ARCH + common_inc
        cmd = [c for c in cmd if c != "--use_fast_math=false"]
        jobs.append((obj, cmd))
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = ["g++", "-c", src, "-o", obj, "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function",
               "-I", os.path.join(cuda, "include")] + common_inc
        jobs.append((obj, cmd))

    def run(job):
        obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stderr.strip() or r.stdout.strip()):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
