"""Build liblbm.so (the C ABIs of include/lbm.h and include/lbm_nn.h) for sm_103a with nvcc, in-tree.

Translation units compile in parallel (one per lattice and storage type plus the runtime) and
are linked into paper_2502_12955_gb300/_build/liblbm.so.  A rebuild happens only when a source
or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fno-strict-aliasing", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
            + [__file__])


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          csrc: str | None = None, out_dir: str | None = None, extra_flags=()) -> str:
    """Compile every CUDA translation unit and link liblbm.so; returns its path.  csrc /
    out_dir / extra_flags build a variant of the sources into another directory."""
    if csrc or out_dir or extra_flags:
        return _build_variant(csrc or CSRC, out_dir or BUILD, list(extra_flags), jobs)
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale(LIB, _deps()):
        return LIB
    nvcc = _nvcc()
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    objs, cmds = [], []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, __file__] + headers):
            cmds.append((obj, [nvcc, *ARCH, *NVFLAGS, "-c", src, "-o", obj + ".tmp"]))
    jobs = jobs or max(1, min(len(cmds), os.cpu_count() or 4))

    def run(item):
        obj, cmd = item
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr[-4000:]}")
        os.replace(obj + ".tmp", obj)
        return r.stderr if verbose else ""

    if cmds:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            for msg in ex.map(run, cmds):
                if msg:
                    print(msg)
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


def _build_variant(csrc, out_dir, extra, jobs):
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(csrc, "*.cu")))
    objs = [os.path.join(out_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    cmds = [[nvcc, *ARCH, *NVFLAGS, *extra, "-c", s, "-o", o] for s, o in zip(srcs, objs)]
    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        for r in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds):
            if r.returncode != 0:
                raise RuntimeError(r.stderr[-4000:])
    lib = os.path.join(out_dir, "liblbm.so")
    r = subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", lib, *objs],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-4000:])
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
