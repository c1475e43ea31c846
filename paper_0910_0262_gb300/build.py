"""Build libqcd.so (the CUDA library behind include/qcd.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked as a shared
library with the shared CUDA runtime (so it shares one runtime with PyTorch).
A stamp of the sources' contents and the flags skips the rebuild when nothing
changed.

    python -m paper_0910_0262_gb300.build          # build if needed
    python -m paper_0910_0262_gb300.build --force  # rebuild
"""

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqcd.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                "-I" + INCLUDE, "-I" + CSRC]
LINK = ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stamp():
    h = hashlib.sha256()
    for d, names in ((CSRC, sorted(os.listdir(CSRC))), (INCLUDE, sorted(os.listdir(INCLUDE)))):
        for n in names:
            p = os.path.join(d, n)
            if os.path.isfile(p):
                h.update(n.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    h.update(" ".join(FLAGS + LINK).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    return r.returncode, r.stdout


def build(force=False, verbose=False, extra_flags=()):
    """Compile every .cu under csrc/ and link libqcd.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp_file = os.path.join(BUILD, "stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return LIB
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([NVCC] + FLAGS + list(extra_flags) + ["-c", os.path.join(CSRC, src), "-o", obj])
    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 4)) as ex:
        results = list(ex.map(_run, cmds))
    for cmd, (rc, out) in zip(cmds, results):
        if verbose or rc:
            sys.stderr.write(" ".join(cmd) + "\n" + out)
        if rc:
            raise RuntimeError("nvcc failed for " + cmd[-3])
    tmp = LIB + ".tmp"
    rc, out = _run([NVCC] + LINK + objs + ["-o", tmp])
    if rc:
        sys.stderr.write(out)
        raise RuntimeError("link of libqcd.so failed")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
