"""Builds libldp.so (all CUDA sources, sm_103a) in-tree.

Translation units are compiled in parallel: the common kernels, the C-ABI,
and the tile-variant kernels (one object per entry of LDP_VARIANTS in
csrc/ldp_launch.h).  Objects go to _build/, the library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import os
import re
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libldp.so")
# checked build (-DLDP_CHECKED): every tile-loop index tested against its buffer
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libldp_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def variants() -> list[tuple[int, int, int, int, int, int]]:
    """(id, rows per tile, warps per CTA, min CTAs per SM, staged, split) of every tile variant
    (split: 1 = narrow tiles split their rows, 2 = histogram slots per region row)."""
    with open(os.path.join(CSRC, "ldp_launch.h")) as f:
        src = f.read()
    m = re.search(r"#define LDP_VARIANTS\(X\)((?:.*\\\n)*.*)", src)
    if not m:
        raise RuntimeError("LDP_VARIANTS not found")
    return [tuple(int(v) for v in t)
            for t in re.findall(r"X\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", m.group(1))]


def _sources_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "ldp.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _compile(args: list[str]) -> tuple[list[str], int, str]:
    p = subprocess.run(args, capture_output=True, text=True)
    return args, p.returncode, p.stdout + p.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, checked: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link libldp.so
    (checked=True: libldp_checked.so with -DLDP_CHECKED, in its own folder).

    Processes that build at the same time (one per rank, parallel test
    workers) take turns on a lock file; a process that waited finds the
    library fresh and returns."""
    bdir = BUILD_CHECKED if checked else BUILD
    os.makedirs(bdir, exist_ok=True)
    with open(os.path.join(bdir, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(force, verbose, jobs, checked)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(force: bool, verbose: bool, jobs: int | None, checked: bool) -> str:
    lib, bdir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    extra = ["-DLDP_CHECKED"] if checked else []
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _sources_mtime():
        return lib
    cc = nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    units = [
        (os.path.join(CSRC, "ldp_common.cu"), os.path.join(bdir, "ldp_common.o"), []),
        (os.path.join(CSRC, "ldp_abi.cu"), os.path.join(bdir, "ldp_abi.o"), []),
        (os.path.join(CSRC, "ldp_noalloc.cu"), os.path.join(bdir, "ldp_noalloc.o"), []),
        (os.path.join(CSRC, "ldp_server.cu"), os.path.join(bdir, "ldp_server.o"), []),
        (os.path.join(CSRC, "ldp_windows.cu"), os.path.join(bdir, "ldp_windows.o"), []),
        (os.path.join(CSRC, "ldp_resize.cu"), os.path.join(bdir, "ldp_resize.o"), []),
        (os.path.join(CSRC, "ldp_distance.cu"), os.path.join(bdir, "ldp_distance.o"), []),
        (os.path.join(CSRC, "ldp_pipeline.cu"), os.path.join(bdir, "ldp_pipeline.o"), []),
    ]
    for vid, rpw, nw, mb, st, sp in variants():
        units.append((os.path.join(CSRC, "ldp_kernels.cu"), os.path.join(bdir, f"ldp_kernels_v{vid}.o"),
                      [f"-DLDP_VAR_ID={vid}", f"-DLDP_VAR_RPW={rpw}", f"-DLDP_VAR_NW={nw}", f"-DLDP_VAR_MB={mb}",
                       f"-DLDP_VAR_ST={st}", f"-DLDP_VAR_SP={sp}"]))
    # the kernels of the other Eq. 2-3 readings (kernel modes 2..4, one unit
    # each), in the tile shape of variant 0
    v0 = variants()[0]
    for cm in (2, 3, 4):
        units.append((os.path.join(CSRC, "ldp_kernels.cu"), os.path.join(bdir, f"ldp_kernels_vcm{cm}.o"),
                      [f"-DLDP_VAR_ID=cm{cm}", f"-DLDP_VAR_RPW={v0[1]}", f"-DLDP_VAR_NW={v0[2]}",
                       f"-DLDP_VAR_MB={v0[3]}", f"-DLDP_VAR_ST={v0[4]}", f"-DLDP_VAR_SP={v0[5]}",
                       f"-DLDP_CODE_MODES={cm}"]))
    cmds = [[cc] + ARCH + FLAGS + extra + inc + defs + ["-c", src, "-o", obj] for src, obj, defs in units]
    jobs = jobs or max(1, min(len(cmds), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(_compile, cmds))
    for args, rc, out in results:
        if rc != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(args) + "\n" + out)
        if verbose and out.strip():
            print(out)
    tmp = lib + f".{os.getpid()}.tmp"
    link = [cc] + ARCH + ["-shared", "-o", tmp] + [obj for _, obj, _ in units]
    p = subprocess.run(link, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + p.stdout + p.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
