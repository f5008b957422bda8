"""Build the in-tree CUDA library libchemgb.so for sm_103a with nvcc.

The library is compiled from paper_2510_10005_gb300/csrc into
paper_2510_10005_gb300/_build/ (git-ignored). Translation units compile in
parallel (instances.cu once per team size and Newton-matrix type, as many
at a time as there are cores); nothing is installed outside the tree.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libchemgb.so")
# the debug build (CG_DEBUG: guard words and poisoned working memory, checked
# after every cell; one-warp teams only), for tests that look for memory errors
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libchemgb_debug.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


# instances.cu is compiled once per team size and Newton-matrix type
INSTANCES = [(team, mt) for team in (32, 64, 128, 256) for mt in ("double", "float")]


def _sources():
    return sorted(p for p in glob.glob(os.path.join(CSRC, "*.cu")) if os.path.basename(p) != "instances.cu")


def _jobs(debug: bool = False):
    """(command, object) of every translation unit, slowest first."""
    jobs = []
    out = BUILD_DEBUG if debug else BUILD
    flags = NVCC_FLAGS + (["-DCG_DEBUG=1"] if debug else [])
    inst = os.path.join(CSRC, "instances.cu")
    for team, mt in INSTANCES:
        if debug and team != 32:
            continue
        obj = os.path.join(out, f"instances_t{team}_{'f64' if mt == 'double' else 'f32'}.o")
        defs = [f"-DCG_TEAM={team}", f"-DCG_MT={mt}", f"-DCG_MT_F64={1 if mt == 'double' else 0}"]
        jobs.append((flags + defs + ["-c", inst, "-o", obj], obj))
    for src in _sources():
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        jobs.append((flags + ["-c", src, "-o", obj], obj))
    return jobs


def _deps():
    return glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(INCLUDE, "*.h"))


def is_stale(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and not is_stale(debug):
        return lib
    os.makedirs(BUILD_DEBUG if debug else BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = _jobs(debug)
    objs = [obj for _, obj in jobs]
    # an object is rebuilt when it is older than its source or any header
    headers = [p for p in _deps() if not p.endswith(".cu")]
    newest_header = max([os.path.getmtime(p) for p in headers] + [0.0])
    def fresh(flags, obj):
        src = flags[flags.index("-c") + 1]
        return (not force and os.path.exists(obj)
                and os.path.getmtime(obj) > max(newest_header, os.path.getmtime(src)))
    width = max(1, os.cpu_count() or 1)
    running, pending = [], [j for j in jobs if not fresh(*j)]
    while pending or running:
        while pending and len(running) < width:
            flags, _ = pending.pop(0)
            cmd = [nvcc] + flags
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            running.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        cmd, p = running.pop(0)
        out, _ = p.communicate()
        if p.returncode != 0:
            for _, q in running:
                q.kill()
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode(errors="replace"))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
