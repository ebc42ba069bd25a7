"""Builds libcontact.so in-tree (paper_2401_10878_gb300/_build/) with nvcc for sm_103a.

Each .cu translation unit is compiled in parallel, then linked into one shared
library with the static CUDA runtime.  Host code is compiled with FP
contraction off: the AABB node ranges are compared bit for bit with an
independent CPU evaluation.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcontact.so")
# the checked build: every index read from a device list is tested
# (-DCONTACT_CHECKS; a failed test sets CONTACT_EBOUNDS and skips the access)
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(BUILD_CHECKS, "libcontact_checks.so")
SOURCES = ["host.cu", "k_broad.cu", "k_narrow.cu", "k_boxmode.cu", "k_post.cu", "k_adjoint.cu", "noalloc.cu",
           "k_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcontact")


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                   "-I", os.path.join(HERE, "..", "include"), *extra]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), checks: bool = False) -> str:
    """Compile (if sources changed) and return the path of libcontact.so, or
    with checks=True of the checked build libcontact_checks.so."""
    out_dir, lib = (BUILD_CHECKS, LIB_CHECKS) if checks else (BUILD, LIB)
    if checks:
        extra_flags = tuple(extra_flags) + ("-DCONTACT_CHECKS",)
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, "contact_dev.cuh"), os.path.join(CSRC, "force_law.cuh"),
               os.path.join(CSRC, "line_clip.cuh"),
               os.path.join(HERE, "..", "include", "contact.h")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [nvcc(), "-c", s, "-o", o + ".tmp"] + flags(extra_flags)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stderr

    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for log in ex.map(compile_one, jobs):
                if verbose and log:
                    print(log)
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, extra_flags=("-Xptxas", "-v")))
