"""Builds libtqr.so (the CUDA library behind include/tqr.h) in-tree with nvcc.

Every translation unit is compiled for sm_103a only, in parallel; objects go to
``_build/`` inside the package and the library to ``libtqr.so`` beside this
file.  ``exec_inst.cu`` is compiled once per executor instantiation (G, PREC)
so that the nine persistent-executor kernels compile in parallel.  A source
newer than the library triggers a rebuild.
"""

import concurrent.futures
import fcntl
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtqr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtqr")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


EXEC_INST = "exec_inst.cu"
EXEC_PAIRS = [(g, p) for g in (4, 8, 16) for p in (0, 1, 2)]


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(os.path.dirname(HERE), "include", "tqr.h"))
    return hs


# ELF e_machine codes of the hosts the library is built on.
_ELF_MACHINE = {"x86_64": 62, "aarch64": 183}


def _lib_matches_host():
    """False when LIB is an ELF file for another CPU than this one (a copy of
    the tree moved between an x86 and an Arm machine)."""
    import platform
    want = _ELF_MACHINE.get(platform.machine())
    try:
        with open(LIB, "rb") as fh:
            head = fh.read(20)
    except OSError:
        return False
    if len(head) < 20 or head[:4] != b"\x7fELF":
        return False
    return want is None or int.from_bytes(head[18:20], "little") == want


def needs_build():
    if not os.path.exists(LIB) or not _lib_matches_host():
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in sources() + _headers() + [__file__])


def build(force=False, verbose=False, extra_flags=()):
    """Compile libtqr.so; returns its path.  Processes that build at the same
    time take turns (a file lock in the build folder); the one that comes
    second finds the library up to date."""
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        try:
            fcntl.flock(lock, fcntl.LOCK_EX)
        except OSError:
            pass                        # a file system without locks: build unserialized
        if not force and not needs_build():
            return LIB
        return _build(verbose, extra_flags)


def _build(verbose, extra_flags):
    nvcc = _nvcc()
    jobs = []
    for src in sources():
        if os.path.basename(src) == EXEC_INST:
            for g, p in EXEC_PAIRS:
                obj = os.path.join(BUILD, "exec_g%d_p%d.o" % (g, p))
                cmd = ([nvcc, "-c", src, "-o", obj, "-DTQR_G=%d" % g, "-DTQR_PREC=%d" % p] + ARCH + FLAGS
                       + list(extra_flags))
                jobs.append((cmd, obj))
            continue
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, "-c", src, "-o", obj] + ARCH + FLAGS + list(extra_flags)
        jobs.append((cmd, obj))

    def run(job):
        cmd, obj = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True, extra_flags=("-Xptxas", "-v")))
