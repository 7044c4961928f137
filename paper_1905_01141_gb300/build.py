"""Build the library: every CUDA translation unit of ``csrc/`` is compiled for
sm_103a in parallel and linked into ``_build/libcrnt.so`` (in-tree), then the
serving load generator ``_build/crnt_loadgen`` (a host program that uses the
library through its C ABI) is linked against it.  The integer issue-rate
probe behind the decode kernel's roofline is a measurement tool and goes into
its own ``_build/libcrnt_probe.so``."""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcrnt.so")
LOADGEN = os.path.join(OUT, "crnt_loadgen")
PROBE = os.path.join(OUT, "libcrnt_probe.so")
UNITS = ["decode.cu", "encode.cu", "crnt_api.cu", "serve.cu", "noalloc.cu", "tune.cu",
         "pusch.cu"]
PROBE_UNIT = "peak.cu"
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v"]


def _units():
    return [u for u in UNITS if os.path.exists(os.path.join(SRC, u))]


def _deps():
    return [os.path.join(SRC, f) for f in os.listdir(SRC)] + [
        os.path.join(HERE, "..", "include", "crnt.h"), os.path.abspath(__file__)]


def up_to_date():
    if not all(os.path.exists(p) for p in (LIB, LOADGEN, PROBE)):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps() if os.path.exists(d))


def _compile(unit):
    obj = os.path.join(OUT, unit + ".o")
    cmd = [NVCC] + FLAGS + ["-c", os.path.join(SRC, unit), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return unit, obj, r.returncode, r.stdout + r.stderr


def _link(out, objs):
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = [NVCC, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs + \
        ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link of %s failed" % os.path.basename(out))
    os.replace(tmp, out)


def build(force=False, verbose=False):
    """Compile and link; returns the path of the shared library."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    units = _units()
    with cf.ThreadPoolExecutor(max_workers=len(units) + 1) as ex:
        res = list(ex.map(_compile, units + [PROBE_UNIT]))
    for unit, obj, rc, log in res:
        if verbose or rc:
            sys.stderr.write(log)
        if rc:
            raise RuntimeError("nvcc failed on %s" % unit)
    objs = {unit: obj for unit, obj, _, _ in res}
    _link(PROBE, [objs[PROBE_UNIT]])
    _link(LIB, [objs[u] for u in units])
    # the serving load generator: a host-only client of the C ABI
    tmp = LOADGEN + ".%d.tmp" % os.getpid()
    cmd = [NVCC, "-O2", "-std=c++17", "-o", tmp, os.path.join(SRC, "loadgen.cpp"), "-L" + OUT,
           "-lcrnt", "-Xlinker", "-rpath,$ORIGIN", "-Xcompiler", "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("loadgen build failed")
    os.replace(tmp, LOADGEN)
    return LIB


def load_probe():
    """The issue-rate probe library (ctypes), built by ``build()``."""
    import ctypes
    L = ctypes.CDLL(PROBE)
    L.crnt_int_issue_probe.restype = ctypes.c_int
    L.crnt_int_issue_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return L


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
