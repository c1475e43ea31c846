"""Build libqcd.so (the CUDA library behind include/qcd.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked as a shared
library with the shared CUDA runtime (so it shares one runtime with PyTorch).
A stamp of the sources' contents and the flags skips the rebuild when nothing
changed.

    python -m paper_0910_0262_gb300.build          # build if needed
    python -m paper_0910_0262_gb300.build --force  # rebuild
    python -m paper_0910_0262_gb300.build --debug  # libqcd_debug.so: index checks in every kernel
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
# the debug build (index checks in every field accessor, reported by qcd_debug_violations)
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libqcd_debug.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                "-I" + INCLUDE, "-I" + CSRC]
LINK = ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stamp(extra=()):
    h = hashlib.sha256()
    for d, names in ((CSRC, sorted(os.listdir(CSRC))), (INCLUDE, sorted(os.listdir(INCLUDE)))):
        for n in names:
            p = os.path.join(d, n)
            if os.path.isfile(p):
                h.update(n.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    h.update(" ".join(FLAGS + list(extra) + LINK).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    return r.returncode, r.stdout


def build(force=False, verbose=False, extra_flags=(), debug=False):
    """Compile every .cu under csrc/ and link libqcd.so (debug: libqcd_debug.so, with QCD_DEBUG=1);
    returns the library path."""
    build_dir = BUILD_DEBUG if debug else BUILD
    lib_path = LIB_DEBUG if debug else LIB
    extra = list(extra_flags) + (["-DQCD_DEBUG=1"] if debug else [])
    os.makedirs(build_dir, exist_ok=True)
    stamp_file = os.path.join(build_dir, "stamp")
    stamp = _stamp(extra)
    if not force and os.path.exists(lib_path) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return lib_path
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([NVCC] + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj])
    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 4)) as ex:
        results = list(ex.map(_run, cmds))
    for cmd, (rc, out) in zip(cmds, results):
        if verbose or rc:
            sys.stderr.write(" ".join(cmd) + "\n" + out)
        if rc:
            raise RuntimeError("nvcc failed for " + cmd[-3])
    tmp = lib_path + ".tmp"
    rc, out = _run([NVCC] + LINK + objs + ["-o", tmp])
    if rc:
        sys.stderr.write(out)
        raise RuntimeError("link of " + os.path.basename(lib_path) + " failed")
    os.replace(tmp, lib_path)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
