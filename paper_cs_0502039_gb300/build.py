"""Build libac.so in-tree for GB300 (sm_103a) with nvcc.

The translation units (kernels, host runtime, allocation-free entry, time-only model) are
compiled in parallel and linked into ``paper_cs_0502039_gb300/libac.so`` (cudart linked
statically).  The same sources are also built with ``-DAC_CHECK`` into ``libac_check.so``:
the bounds-checked variant whose kernels check every index they compute and report a
violation as AC_ERR_STATE (the tests load it in a subprocess through AC_LIB_PATH).
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libac.so")
LIB_CHECK = os.path.join(PKG, "libac_check.so")
SOURCES = ["ac_kernels.cu", "ac_api.cu", "ac_static.cu", "ac_time.cu"]
HEADERS = ["ac_device.cuh", "ac_internal.h"]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I", INCLUDE, "-I", CSRC]
VARIANTS = ((LIB, os.path.join(PKG, "_build"), []), (LIB_CHECK, os.path.join(PKG, "_build_check"), ["-DAC_CHECK"]))


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "ac.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    todo = [v for v in VARIANTS if force or _stale(v[0])]
    if not todo:
        return LIB
    nvcc = _nvcc()
    procs = []
    for lib, bdir, extra in todo:
        os.makedirs(bdir, exist_ok=True)
        for src in SOURCES:
            obj = os.path.join(bdir, src.replace(".cu", ".o"))
            cmd = [nvcc, *extra, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    for lib, bdir, _ in todo:
        objs = [os.path.join(bdir, src.replace(".cu", ".o")) for src in SOURCES]
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", *objs, "-o", tmp], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
