"""ctypes wrapper of oracle/capply.c: the modified adjoint NFFT D^* F^* B_opt^* f
(eq:approx_ansatz2) on the CPU in plain C with OpenMP (gather, radix-2 FFT, D), given the
oracle's B_opt.  Test infrastructure: an independent second evaluation of the oracle's numpy
apply, and the multi-core CPU baseline of the benchmark.  build() compiles it with gcc."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "capply.c")
LIB = os.path.join(HERE, "_build", "libcapply.so")
_lib = None


def build(force=False):
    """Compiles capply.c into oracle/_build/libcapply.so (gcc, OpenMP); returns the path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed on capply.c:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def library():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        for name in ("capply_f64", "capply_f32"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P, P]
            fn.restype = ctypes.c_int
        lib.capply_twiddles.argtypes = [ctypes.c_int64, P]
        lib.capply_twiddles.restype = None
        lib.capply_threads.argtypes = []
        lib.capply_threads.restype = ctypes.c_int
        lib.capply_set_threads.argtypes = [ctypes.c_int]
        lib.capply_set_threads.restype = None
        _lib = lib
    return _lib


def threads():
    """OpenMP threads the C apply runs on."""
    return int(library().capply_threads())


def set_threads(n):
    """Sets the OpenMP threads of the following C applies."""
    library().capply_set_threads(int(n))


class CApply:
    """B_opt of the oracle (oracle.bopt.BOpt) prepared for the C apply; __call__(f) -> fhat."""

    def __init__(self, B, precision="f64"):
        self.B = B
        self.real = np.float64 if precision == "f64" else np.float32
        self.ptr = np.ascontiguousarray(B.ptr, np.int64)
        self.idx = np.ascontiguousarray(B.idx, np.int64)
        self.b = np.ascontiguousarray(B.b, np.float64)
        self.tw = np.empty(B.Ms, np.float64)
        library().capply_twiddles(B.Ms, self.tw.ctypes.data)
        self.work = np.empty(2 * B.Ms, self.real)
        self.fn = library().capply_f64 if precision == "f64" else library().capply_f32

    def __call__(self, f, out=None):
        cplx = np.complex128 if self.real is np.float64 else np.complex64
        f = np.ascontiguousarray(f, cplx)
        if out is None:
            out = np.empty(self.B.M, cplx)
        rc = self.fn(self.B.Ms, self.B.M, 1 if self.B.kernel == "sym" else 0, self.ptr.ctypes.data,
                     self.idx.ctypes.data, self.b.ctypes.data, f.ctypes.data, out.ctypes.data,
                     self.work.ctypes.data, self.tw.ctypes.data)
        if rc != 0:
            raise ValueError("capply: M_sigma must be a power of two and M even, M <= M_sigma")
        return out
