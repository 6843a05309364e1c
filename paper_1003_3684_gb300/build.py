"""Build libpgen.so (the CUDA library behind include/pgen.h) in-tree.

Compiles every csrc/*.cu for sm_103a in parallel with nvcc and links them
into paper_1003_3684_gb300/libpgen.so (CUDA runtime linked statically, so the
library only needs the NVIDIA driver). The same sources compiled with -DPGEN_CHECKED
give libpgen_checked.so, the bounds-checked build (the same entry points;
pg_check_read reports what its checks found). Run
``python -m paper_1003_3684_gb300.build`` (``--force`` rebuilds everything).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--extended-lambda", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-Wall"]
# variant -> (library, object folder, extra flags)
VARIANTS = {
    "default": ("libpgen.so", "_build", []),
    "checked": ("libpgen_checked.so", "_build_checked", ["-DPGEN_CHECKED"]),
}
OUT = os.path.join(HERE, VARIANTS["default"][0])


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the pgen CUDA library cannot be built")


def _stale(obj: str, deps: list[str]) -> bool:
    return not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(d) for d in deps)


def _run(cmd: list[str], verbose: bool) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr)


def build(force: bool = False, verbose: bool = False,
          variants: tuple[str, ...] = ("default", "checked")) -> str:
    """Compile the requested variants (all translation units of all variants
    in one parallel pool), link each library, and return the default one's
    path."""
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                     glob.glob(os.path.join(HERE, "..", "include", "*.h")))
    plans = []   # (library path, objects, any object rebuilt)
    jobs = []
    for name in variants:
        lib, folder, extra = VARIANTS[name]
        obj_dir = os.path.join(HERE, folder)
        os.makedirs(obj_dir, exist_ok=True)
        objs = []
        fresh = False
        for src in sources:
            obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                jobs.append([nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj])
                fresh = True
        plans.append((os.path.join(HERE, lib), objs, fresh))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(lambda c: _run(c, verbose), jobs))
    for lib, objs, fresh in plans:
        if force or fresh or not os.path.exists(lib) or _stale(lib, objs):
            tmp = lib + f".tmp{os.getpid()}"
            _run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs, verbose)
            os.replace(tmp, lib)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
