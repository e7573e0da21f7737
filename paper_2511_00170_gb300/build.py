"""Build the engine's shared library (libah.so) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into ``libah.so`` next to
this file.  The scan kernel itself is specialised per primer set at run time with NVRTC (linked
here), so only the fixed kernels are compiled now.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libah.so")
SOURCES = ["ah_api.cu", "ah_util.cu", "ah_scan.cu", "ah_pair.cu", "ah_tm.cu", "ah_extract.cu", "ah_plan.cu", "ah_fasta.cu", "ah_jit.cpp",
           "ah_tm_jit.cpp", "ah_serve.cpp", "ah_output.cpp", "ah_files.cpp"]
# headers every translation unit may include; ah_tm_chain.cuh is also compiled at run time (its text
# is embedded in the library by _embed)
HEADERS = ["ah_internal.h", "ah_tm_chain.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, *(os.path.join(CSRC, h) for h in HEADERS), os.path.join(HERE, "..", "include", "ah.h")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps if os.path.exists(d))


def _embed(header: str, out: str) -> None:
    """Write header's text as a C++ raw string literal (rewritten only when it changes)."""
    with open(header) as f:
        text = f.read()
    assert ")AHSRC\"" not in text
    lit = 'R"AHSRC(' + text + ')AHSRC"\n'
    if os.path.exists(out):
        with open(out) as f:
            if f.read() == lit:
                return
    with open(out + ".tmp", "w") as f:
        f.write(lit)
    os.replace(out + ".tmp", out)


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    cuda = _cuda_home(nvcc)
    os.makedirs(BUILD, exist_ok=True)
    _embed(os.path.join(CSRC, "ah_tm_chain.cuh"), os.path.join(BUILD, "ah_tm_chain_src.inc"))
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(HERE, "..", "include"),
              "-I", BUILD]
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        if force or _stale(obj, src):
            lang = [] if s.endswith(".cu") else ["-x", "cu"]
            jobs.append([nvcc, *ARCH, *common, *lang, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, s + ".o") for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        libdirs = [os.path.join(cuda, "lib64"), os.path.join(cuda, "lib64", "stubs"),
                   os.path.join(cuda, "targets", "sbsa-linux", "lib"), os.path.join(cuda, "targets", "x86_64-linux", "lib")]
        link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        for d in libdirs:
            if os.path.isdir(d):
                link += ["-L", d]
        link += ["-lnvrtc", "-Xlinker", "-rpath," + os.path.join(cuda, "lib64")]
        run(link)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
