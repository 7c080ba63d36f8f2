"""Build step of the CUDA library (librf.so, sm_103a) — run by
``__graft_entry__.build()`` or ``python -m paper_2506_04763_gb300.build``.

Each translation unit is compiled in parallel with nvcc for sm_103a only, and
linked in-tree into ``paper_2506_04763_gb300/librf.so``.  The assembly unit is
compiled with -fmad=false (see the header comment of assemble.cu).
"""
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "librf")
LIB = os.path.join(PKG, "librf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {"assemble.cu": ["-fmad=false"], "levelops.cu": [], "krylov.cu": [], "driver.cu": [], "noalloc.cu": [], "probe.cu": []}


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librf.so")
    return cand


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "rf.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, unit), "-o", obj] + common + extra
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(unit)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call([cc, "-shared", "-o", tmp] + objs + ARCH)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
