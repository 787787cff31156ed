"""Build the CUDA library libsfd.so for sm_103a (in-tree, no cmake).

The host runtime and the per-class step kernels are compiled in parallel
with nvcc and linked into
``paper_2311_18505_gb300/_build/libsfd.so``.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsfd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
# (source, object, extra flags): the step kernel is compiled once per
# transverse rows-per-lane class so each kernel gets its own register budget
UNITS = [("sfd_api.cu", "sfd_api.o", []), ("sfd_adjoint.cu", "sfd_adjoint.o", []),
         ("sfd_peaks.cu", "sfd_peaks.o", [])] + \
        [("sfd_kernel.cu", f"sfd_kernel_r{mu}.o", [f"-DSFD_MU={mu}"]) for mu in (1, 3, 5, 7, 9)] + \
        [("sfd_kernel.cu", "sfd_kernel_smem.o", [])]
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = ["sfd_types.h", "sfd_df64.cuh", "sfd_device.cuh", "sfd_step_reg.cuh", "sfd_step_smem.cuh", "sfd_server.cuh",
           "sfd_tape.cuh"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsfd.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "sfd.h"),
                                                                  os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    procs, objs = [], []
    for src, o, extra in UNITS:
        obj = os.path.join(OUT_DIR, o)
        objs.append(obj)
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{out.decode(errors='replace')}")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", *ARCH, *objs, "-o", tmp]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout.decode(errors='replace')}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
