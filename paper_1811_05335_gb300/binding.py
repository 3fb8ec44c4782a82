"""ctypes binding of libinfft_gb300.so (same names as the C ABI in include/infft.h).

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they are passed to the
library as raw pointers (the library detects host vs device memory).  Complex data
is complex64 (infft_apply / nfft_apply) or complex128 (the _z variants); nodes
are float64.  ``stream`` is a torch.cuda.Stream, a raw cudaStream_t integer, or
None for torch's current stream when a CUDA tensor is involved (else the legacy
default stream)."""
import ctypes
import os

import numpy as np

from . import build as _build

KERNEL_FULL, KERNEL_SYM = 0, 1
_KERNELS = {"full": KERNEL_FULL, "sym": KERNEL_SYM, KERNEL_FULL: KERNEL_FULL, KERNEL_SYM: KERNEL_SYM}
_STATUS = {0: "INFFT_OK", 1: "INFFT_EINVAL", 2: "INFFT_ENOMEM", 3: "INFFT_ECUDA", 4: "INFFT_ENOTREADY",
           5: "INFFT_EUNSUPPORTED", 6: "INFFT_ENUMERIC"}

EXPORTED_SYMBOLS = (
    "infft_plan", "infft_precompute", "infft_apply", "nfft_apply", "plan_destroy", "infft_plan_create",
    "infft_set_nodes", "infft_apply_z", "nfft_apply_z", "infft_get_info", "infft_copy_plan_data",
    "infft_profile", "infft_profile_read", "infft_launch_count", "infft_last_error", "infft_version",
    "infft_fft_deconv_noalloc", "infft_grad_nodes", "infft_plan_create_ansatz",
    "infft_batch_create", "infft_batch_set_nodes", "infft_batch_precompute", "infft_batch_apply",
    "infft_batch_get_info", "infft_batch_copy_problem", "infft_batch_destroy",
    "infft_apply_many", "infft_apply_many_workspace",
    "infft2d_plan_create", "infft2d_set_nodes", "infft2d_precompute", "infft2d_apply", "infft2d_apply_z",
    "infft2d_get_info", "infft2d_copy_plan_data", "infft2d_plan_destroy",
    "infft_ndft_z", "infft_refine_z", "infft_nfft_kb_z",
    "infft_apply_sorted", "infft_sort_values", "infft_apply_config_count", "infft_apply_config_shape",
    "infft_set_apply_config", "infft_get_apply_config", "infft_tune_apply",
    "infft_fp64_fma_probe", "infft_fp64_fma_probe_sink_len",
    "infft_batch_tile_shape_count", "infft_batch_tile_shape", "infft_batch_set_tile_shape",
    "infft_batch_get_tile_shape", "infft_batch_tune_apply",
)


class InfftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class _Info(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("M_sigma", ctypes.c_int64),
                ("m", ctypes.c_int32), ("kernel", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("tau", ctypes.c_double), ("nnz", ctypes.c_int64), ("max_column", ctypes.c_int32),
                ("empty_columns", ctypes.c_int32), ("bad_nodes", ctypes.c_int32),
                ("fallback_columns", ctypes.c_int32), ("unsupported_columns", ctypes.c_int32),
                ("nodes_set", ctypes.c_int32), ("precomputed", ctypes.c_int32), ("objective", ctypes.c_double),
                ("grad_failed_columns", ctypes.c_int32), ("ansatz", ctypes.c_int32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int64), ("sum_N", ctypes.c_int64), ("sum_M", ctypes.c_int64),
                ("m", ctypes.c_int32), ("nodes_set", ctypes.c_int32), ("precomputed", ctypes.c_int32),
                ("max_column", ctypes.c_int32), ("nnz", ctypes.c_int64), ("empty_columns", ctypes.c_int64),
                ("bad_nodes", ctypes.c_int64), ("fallback_columns", ctypes.c_int64),
                ("unsupported_columns", ctypes.c_int64), ("large_columns", ctypes.c_int64),
                ("objective", ctypes.c_double)]


class _Info2D(ctypes.Structure):
    _fields_ = [("M1", ctypes.c_int64), ("M2", ctypes.c_int64), ("M_sigma1", ctypes.c_int64),
                ("M_sigma2", ctypes.c_int64), ("N", ctypes.c_int64), ("m", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("sigma", ctypes.c_double), ("tau", ctypes.c_double),
                ("nnz", ctypes.c_int64), ("max_column", ctypes.c_int32), ("empty_columns", ctypes.c_int32),
                ("bad_nodes", ctypes.c_int32), ("fallback_columns", ctypes.c_int32),
                ("unsupported_columns", ctypes.c_int32), ("large_columns", ctypes.c_int32),
                ("wide_columns", ctypes.c_int32), ("nodes_set", ctypes.c_int32), ("precomputed", ctypes.c_int32),
                ("objective", ctypes.c_double), ("indexed_columns", ctypes.c_int32)]


_lib = None


def library():
    """Loads the built library (raises InfftError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.lib_path()
    if not os.path.exists(path):
        raise InfftError(-1, f"{path} is not built; run __graft_entry__.build() (needs nvcc)")
    lib = ctypes.CDLL(path)
    P, I64, I32, D, VP = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "infft_plan": [I64, I64, VP, D, I32, ctypes.POINTER(P)],
        "infft_plan_create": [I64, I64, D, I32, I32, D, ctypes.POINTER(P)],
        "infft_plan_create_ansatz": [I64, I64, D, I32, I32, I32, D, ctypes.POINTER(P)],
        "infft_set_nodes": [P, VP, VP],
        "infft_precompute": [P, VP],
        "infft_apply": [P, VP, VP, VP],
        "nfft_apply": [P, VP, VP, VP],
        "infft_apply_z": [P, VP, VP, VP],
        "nfft_apply_z": [P, VP, VP, VP],
        "plan_destroy": [P],
        "infft_get_info": [P, ctypes.POINTER(_Info)],
        "infft_copy_plan_data": [P, VP, VP, VP, VP, VP, VP],
        "infft_profile": [P, I32],
        "infft_fft_deconv_noalloc": [VP, I64, I64, I32, VP, VP],
        "infft_grad_nodes": [P, VP, VP, VP, VP],
        "infft_profile_read": [P, I32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(I64),
                               ctypes.POINTER(D), ctypes.POINTER(I32)],
        "infft_batch_create": [I64, VP, VP, D, I32, I32, D, ctypes.POINTER(P)],
        "infft_batch_set_nodes": [P, VP, VP],
        "infft_batch_precompute": [P, VP],
        "infft_batch_apply": [P, VP, VP, VP],
        "infft_batch_get_info": [P, ctypes.POINTER(_BatchInfo)],
        "infft_batch_copy_problem": [P, I64, VP, VP, VP, VP, VP, VP],
        "infft_batch_destroy": [P],
        "infft_apply_many": [P, I64, VP, VP, VP, I64, VP],
        "infft_ndft_z": [P, VP, VP, VP],
        "infft_refine_z": [P, VP, VP, I32, VP],
        "infft_nfft_kb_z": [P, VP, VP, VP],
        "infft2d_plan_create": [I64, I64, I64, D, I32, I32, D, ctypes.POINTER(P)],
        "infft2d_set_nodes": [P, VP, VP],
        "infft2d_precompute": [P, VP],
        "infft2d_apply": [P, VP, VP, VP],
        "infft2d_apply_z": [P, VP, VP, VP],
        "infft2d_get_info": [P, ctypes.POINTER(_Info2D)],
        "infft2d_copy_plan_data": [P, VP, VP, VP, VP],
        "infft2d_plan_destroy": [P],
        "infft_apply_sorted": [P, VP, VP, VP],
        "infft_sort_values": [P, VP, VP, VP],
        "infft_apply_config_shape": [I32, ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "infft_set_apply_config": [P, I32],
        "infft_tune_apply": [P, I32, VP, ctypes.POINTER(I32), VP],
        "infft_fp64_fma_probe": [I64, VP, I64, ctypes.POINTER(D), VP],
        "infft_batch_tile_shape": [I32, ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "infft_batch_set_tile_shape": [P, I32, VP],
        "infft_batch_tune_apply": [P, I32, VP, ctypes.POINTER(I32), VP],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.infft_apply_many_workspace.restype = ctypes.c_int64
    lib.infft_apply_many_workspace.argtypes = [P, I64]
    lib.infft_fp64_fma_probe_sink_len.restype = ctypes.c_int64
    lib.infft_fp64_fma_probe_sink_len.argtypes = []
    lib.infft_apply_config_count.restype = ctypes.c_int
    lib.infft_apply_config_count.argtypes = []
    lib.infft_get_apply_config.restype = ctypes.c_int
    lib.infft_get_apply_config.argtypes = [P]
    lib.infft_batch_tile_shape_count.restype = ctypes.c_int
    lib.infft_batch_tile_shape_count.argtypes = []
    lib.infft_batch_get_tile_shape.restype = ctypes.c_int
    lib.infft_batch_get_tile_shape.argtypes = [P]
    lib.infft_launch_count.restype = ctypes.c_int64
    lib.infft_launch_count.argtypes = []
    lib.infft_last_error.restype = ctypes.c_char_p
    lib.infft_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code):
    if code != 0:
        raise InfftError(code, library().infft_last_error().decode())


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _as_ptr(a, kind, keep):
    """Raw pointer of a contiguous array of the wanted element kind."""
    if _is_torch(a):
        import torch
        want = {"c64": torch.complex64, "c128": torch.complex128, "f64": torch.float64}[kind]
        if a.dtype != want:
            raise TypeError(f"expected a {want} tensor, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        keep.append(a)
        return a.data_ptr()
    want = {"c64": np.complex64, "c128": np.complex128, "f64": np.float64}[kind]
    arr = np.ascontiguousarray(a, dtype=want)
    keep.append(arr)
    return arr.ctypes.data


def _stream(stream, *arrays):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    for a in arrays:
        if _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return 0


def _empty_like(ref, n, kind):
    if _is_torch(ref):
        import torch
        dt = {"c64": torch.complex64, "c128": torch.complex128}[kind]
        return torch.empty(n, dtype=dt, device=ref.device)
    return np.empty(n, dtype={"c64": np.complex64, "c128": np.complex128}[kind])


class Plan:
    """Owner of an infft_plan_t handle (released by plan_destroy or close())."""

    def __init__(self, handle, M, N, Ms, m):
        self.handle, self.M, self.N, self.M_sigma, self.m = handle, M, N, Ms, m

    def close(self):
        if self.handle:
            _check(library().plan_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ms(M, sigma):
    return int(round(sigma * M))


def infft_plan(M, N, x, sigma, m):
    """Creates a plan for nodes x (kernel full, tau = 1e-12) and runs the pattern step."""
    keep = []
    h = ctypes.c_void_p()
    _check(library().infft_plan(M, N, _as_ptr(x, "f64", keep), float(sigma), int(m), ctypes.byref(h)))
    return Plan(h.value, M, N, _ms(M, sigma), m)


def infft_plan_create(M, N, sigma, m, kernel="full", tau=1e-12):
    h = ctypes.c_void_p()
    k = _KERNELS.get(kernel, kernel) if isinstance(kernel, (str, int)) else kernel
    _check(library().infft_plan_create(M, N, float(sigma), int(m), int(k), float(tau), ctypes.byref(h)))
    return Plan(h.value, M, N, _ms(M, sigma), m)


ANSATZ_UNDERDETERMINED, ANSATZ_OVERDETERMINED = 1, 2
_ANSATZ = {"under": ANSATZ_UNDERDETERMINED, "underdetermined": ANSATZ_UNDERDETERMINED,
           "over": ANSATZ_OVERDETERMINED, "overdetermined": ANSATZ_OVERDETERMINED}


def infft_plan_create_ansatz(M, N, sigma, m, kernel="full", ansatz="over", tau=1e-12):
    """As infft_plan_create with the optimisation of Sec. 3.2.1 ("under") or 3.2.2 ("over")."""
    h = ctypes.c_void_p()
    k = _KERNELS.get(kernel, kernel) if isinstance(kernel, (str, int)) else kernel
    a = _ANSATZ.get(ansatz, ansatz)
    _check(library().infft_plan_create_ansatz(M, N, float(sigma), int(m), int(k), int(a), float(tau),
                                              ctypes.byref(h)))
    plan = Plan(h.value, M, N, _ms(M, sigma), m)
    plan.ansatz = int(a)
    return plan


def infft_set_nodes(plan, x, stream=None):
    keep = []
    _check(library().infft_set_nodes(plan.handle, _as_ptr(x, "f64", keep), _stream(stream, x)))


def infft_precompute(plan, stream=None):
    _check(library().infft_precompute(plan.handle, _stream(stream)))


def _apply(fn, plan, src, out, n_out, kind, stream):
    keep = []
    if out is None:
        out = _empty_like(src, n_out, kind)
    _check(fn(plan.handle, _as_ptr(src, kind, keep), _as_ptr(out, kind, keep), _stream(stream, src, out)))
    return out


def infft_apply(plan, f, out=None, stream=None):
    """fhat = D^* F^* B_opt^* f (complex64)."""
    return _apply(library().infft_apply, plan, f, out, plan.M, "c64", stream)


def nfft_apply(plan, fhat, out=None, stream=None):
    """f = B_opt F D fhat (complex64), the adjoint of infft_apply."""
    return _apply(library().nfft_apply, plan, fhat, out, plan.N, "c64", stream)


def infft_apply_sorted(plan, f_sorted, out=None, stream=None):
    """fhat = D^* F^* B_opt^* f from samples in the plan's sorted node order (complex64, device)."""
    return _apply(library().infft_apply_sorted, plan, f_sorted, out, plan.M, "c64", stream)


def infft_sort_values(plan, f, out=None, stream=None):
    """f_sorted[i] = f[perm[i]] (complex64 device tensors)."""
    return _apply(library().infft_sort_values, plan, f, out, plan.N, "c64", stream)


def infft_apply_configs():
    """[(log2 N1, columns per run)] of every tile shape of the fp32 apply, by id."""
    lib = library()
    out = []
    for i in range(lib.infft_apply_config_count()):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib.infft_apply_config_shape(i, ctypes.byref(a), ctypes.byref(b)))
        out.append((a.value, b.value))
    return out


def infft_set_apply_config(plan, config):
    """Tile shape id for the plan's fp32 apply (-1: the default rule)."""
    _check(library().infft_set_apply_config(plan.handle, int(config)))


def infft_get_apply_config(plan):
    """Tile shape id the next apply uses (-1: the three-launch path)."""
    return int(library().infft_get_apply_config(plan.handle))


def infft_tune_apply(plan, repeats=20, stream=None):
    """Times every valid tile shape on the plan and keeps the fastest: (best id, [ms per id])."""
    lib = library()
    n = lib.infft_apply_config_count()
    ms = (ctypes.c_float * n)()
    best = ctypes.c_int(-1)
    _check(lib.infft_tune_apply(plan.handle, int(repeats), ctypes.cast(ms, ctypes.c_void_p), ctypes.byref(best),
                                _stream(stream)))
    return best.value, [float(v) for v in ms]


def infft_apply_many_workspace(plan, K):
    """Bytes of device workspace infft_apply_many needs for K vectors."""
    return int(library().infft_apply_many_workspace(plan.handle, int(K)))


def infft_apply_many(plan, f, out=None, workspace=None, stream=None):
    """fhat of K data vectors (f: K x N complex64 CUDA tensor) -> K x M complex64."""
    import torch
    keep = []
    K = int(f.shape[0])
    if out is None:
        out = torch.empty((K, plan.M), dtype=torch.complex64, device=f.device)
    need = infft_apply_many_workspace(plan, K)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=f.device)
    _check(library().infft_apply_many(plan.handle, K, _as_ptr(f, "c64", keep), _as_ptr(out, "c64", keep),
                                      workspace.data_ptr(), int(workspace.numel() * workspace.element_size()),
                                      _stream(stream, f, out)))
    return out


def infft_apply_z(plan, f, out=None, stream=None):
    return _apply(library().infft_apply_z, plan, f, out, plan.M, "c128", stream)


def nfft_apply_z(plan, fhat, out=None, stream=None):
    return _apply(library().nfft_apply_z, plan, fhat, out, plan.N, "c128", stream)


def infft_ndft_z(plan, fhat, out=None, stream=None):
    """f = A fhat by the direct fp64 sum at the plan's nodes (device complex128 tensors)."""
    keep = []
    if out is None:
        out = _empty_like(fhat, plan.N, "c128")
    _check(library().infft_ndft_z(plan.handle, _as_ptr(fhat, "c128", keep), _as_ptr(out, "c128", keep),
                                  _stream(stream, fhat, out)))
    return out


def infft_nfft_kb_z(plan, fhat, out=None, stream=None):
    """f ~ A fhat by the windowed fp64 NFFT (Kaiser-Bessel, sigma >= 2; device complex128 tensors)."""
    keep = []
    if out is None:
        out = _empty_like(fhat, plan.N, "c128")
    _check(library().infft_nfft_kb_z(plan.handle, _as_ptr(fhat, "c128", keep), _as_ptr(out, "c128", keep),
                                     _stream(stream, fhat, out)))
    return out


def infft_refine_z(plan, f, fhat, sweeps=1, stream=None):
    """fhat <- fhat + D^* F^* B_opt^* (f - A fhat), `sweeps` times, in place (device complex128)."""
    keep = []
    _check(library().infft_refine_z(plan.handle, _as_ptr(f, "c128", keep), _as_ptr(fhat, "c128", keep),
                                    int(sweeps), _stream(stream, f, fhat)))
    return fhat


def plan_destroy(plan):
    plan.close()


def infft_get_info(plan):
    info = _Info()
    _check(library().infft_get_info(plan.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in _Info._fields_}


def infft_copy_plan_data(plan, weights=True):
    """Pattern and B_opt as host numpy arrays (see include/infft.h)."""
    info = infft_get_info(plan)
    N, Ms, nnz = plan.N, plan.M_sigma, int(info["nnz"])
    perm = np.empty(N, np.int32)
    start = np.empty(Ms, np.int32)
    count = np.empty(Ms, np.int32)
    off = np.empty(Ms + 1, np.int32)
    w = np.empty(max(nnz, 1), np.float64) if weights else None
    nJ = N if info.get("ansatz") == ANSATZ_UNDERDETERMINED else Ms
    J = np.empty(nJ, np.float64) if weights else None
    ptr = lambda a: a.ctypes.data if a is not None else None
    _check(library().infft_copy_plan_data(plan.handle, ptr(perm), ptr(start), ptr(count), ptr(off), ptr(w),
                                          ptr(J)))
    out = dict(perm=perm, col_start=start, col_count=count, col_offset=off)
    if weights:
        out.update(weights=w[:nnz], objective=J)
    return out


def infft_profile(plan, enable=True):
    _check(library().infft_profile(plan.handle, 1 if enable else 0))


def infft_profile_read(plan):
    cap = 64
    names = (ctypes.c_char_p * cap)()
    launches = (ctypes.c_int64 * cap)()
    ms = (ctypes.c_double * cap)()
    n = ctypes.c_int()
    _check(library().infft_profile_read(plan.handle, cap, names, launches, ms, ctypes.byref(n)))
    return [(names[i].decode(), int(launches[i]), float(ms[i])) for i in range(n.value)]


def infft_fft_deconv_noalloc(grid, M, out=None, kernel="full", stream=None):
    """fhat = D^* F^* grid (complex64, device tensors) without any allocation in the
    library (see include/infft.h); `out` is allocated here by torch when not given."""
    import torch
    keep = []
    if out is None:
        out = _empty_like(grid, M, "c64")
    if isinstance(grid, torch.Tensor) and isinstance(out, torch.Tensor) and grid.device != out.device:
        raise InfftError(1, f"grid ({grid.device}) and out ({out.device}) must be on the same device")
    k = _KERNELS.get(kernel, kernel)
    # the library takes its scratch array on the current device: make grid's device current
    with torch.cuda.device(grid.device if isinstance(grid, torch.Tensor) and grid.is_cuda else None):
        _check(library().infft_fft_deconv_noalloc(_as_ptr(grid, "c64", keep), int(M), int(grid.shape[0]), int(k),
                                                  _as_ptr(out, "c64", keep), _stream(stream, grid, out)))
    return out


def infft_grad_nodes(plan, f, w, out=None, stream=None):
    """dL/dx (float64, device) for data f and w = dL/dRe fhat + i dL/dIm fhat (complex64, device)."""
    import torch
    keep = []
    if out is None:
        out = torch.empty(plan.N, dtype=torch.float64, device=f.device)
    _check(library().infft_grad_nodes(plan.handle, _as_ptr(f, "c64", keep), _as_ptr(w, "c64", keep),
                                      _as_ptr(out, "f64", keep), _stream(stream, f, w, out)))
    return out


def infft_fp64_fma_probe(iters, sink, stream=None):
    """Launches the fp64 FMA throughput probe on `stream` (sink: float64 CUDA tensor of at least
    infft_fp64_fma_probe_sink_len() elements); returns the launch's flop count."""
    keep = []
    flops = ctypes.c_double()
    _check(library().infft_fp64_fma_probe(int(iters), _as_ptr(sink, "f64", keep), int(sink.numel()),
                                          ctypes.byref(flops), _stream(stream, sink)))
    return flops.value


def infft_fp64_fma_probe_sink_len():
    return int(library().infft_fp64_fma_probe_sink_len())


def infft_launch_count():
    return int(library().infft_launch_count())


def infft_version():
    return library().infft_version().decode()


class Batch:
    """Owner of an infft_batch_t handle: P independent problems of sizes M[p], N[p]."""

    def __init__(self, handle, M, N, m):
        self.handle, self.M, self.N, self.m = handle, np.asarray(M, np.int64), np.asarray(N, np.int64), m
        self.P = len(self.M)
        self.n_off = np.concatenate([[0], np.cumsum(self.N)])
        self.m_off = np.concatenate([[0], np.cumsum(self.M)])

    def close(self):
        if self.handle:
            _check(library().infft_batch_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def infft_batch_create(M, N, sigma=2.0, m=6, kernel="full", tau=1e-12):
    """Batch of len(M) problems (M[p] coefficients, N[p] nodes), sigma = 2."""
    Ma = np.ascontiguousarray(M, np.int64)
    Na = np.ascontiguousarray(N, np.int64)
    if Ma.shape != Na.shape or Ma.ndim != 1:
        raise ValueError("M and N must be 1-D arrays of the same length")
    h = ctypes.c_void_p()
    k = _KERNELS.get(kernel, kernel)
    _check(library().infft_batch_create(len(Ma), Ma.ctypes.data, Na.ctypes.data, float(sigma), int(m), int(k),
                                        float(tau), ctypes.byref(h)))
    return Batch(h.value, Ma, Na, m)


def infft_batch_set_nodes(batch, x, stream=None):
    keep = []
    _check(library().infft_batch_set_nodes(batch.handle, _as_ptr(x, "f64", keep), _stream(stream, x)))


def infft_batch_precompute(batch, stream=None):
    _check(library().infft_batch_precompute(batch.handle, _stream(stream)))


def infft_batch_apply(batch, f, out=None, stream=None):
    """fhat of every problem (complex64, problems back to back)."""
    keep = []
    if out is None:
        out = _empty_like(f, int(batch.m_off[-1]), "c64")
    _check(library().infft_batch_apply(batch.handle, _as_ptr(f, "c64", keep), _as_ptr(out, "c64", keep),
                                       _stream(stream, f, out)))
    return out


def infft_batch_tile_shapes():
    """[(grid points per tile, weights per block)] of every tile shape of the batched spreading, by id."""
    lib = library()
    out = []
    for i in range(lib.infft_batch_tile_shape_count()):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib.infft_batch_tile_shape(i, ctypes.byref(a), ctypes.byref(b)))
        out.append((a.value, b.value))
    return out


def infft_batch_set_tile_shape(batch, shape, stream=None):
    """Tile shape id of the batched spreading (-1: the fixed default rule)."""
    _check(library().infft_batch_set_tile_shape(batch.handle, int(shape), _stream(stream)))


def infft_batch_get_tile_shape(batch):
    """Tile shape id the next batched apply uses."""
    return int(library().infft_batch_get_tile_shape(batch.handle))


def infft_batch_tune_apply(batch, repeats=10, stream=None):
    """Times every tile shape on the batch and keeps the fastest: (best id, [ms per id])."""
    lib = library()
    n = lib.infft_batch_tile_shape_count()
    ms = (ctypes.c_float * n)()
    best = ctypes.c_int(-1)
    _check(lib.infft_batch_tune_apply(batch.handle, int(repeats), ctypes.cast(ms, ctypes.c_void_p),
                                      ctypes.byref(best), _stream(stream)))
    return best.value, [float(v) for v in ms]


def infft_batch_get_info(batch):
    info = _BatchInfo()
    _check(library().infft_batch_get_info(batch.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in _BatchInfo._fields_}


def infft_batch_copy_problem(batch, p, weights=True):
    """Pattern and B_opt of problem p as host numpy arrays (as infft_copy_plan_data)."""
    N, Ms = int(batch.N[p]), 2 * int(batch.M[p])
    perm = np.empty(N, np.int32)
    start = np.empty(Ms, np.int32)
    count = np.empty(Ms, np.int32)
    off = np.empty(Ms + 1, np.int32)
    ptr = lambda a: a.ctypes.data if a is not None else None
    _check(library().infft_batch_copy_problem(batch.handle, int(p), ptr(perm), ptr(start), ptr(count), ptr(off),
                                              None, None))
    out = dict(perm=perm, col_start=start, col_count=count, col_offset=off)
    if weights:
        nnz = int(off[-1])
        w = np.empty(max(nnz, 1), np.float64)
        J = np.empty(Ms, np.float64)
        _check(library().infft_batch_copy_problem(batch.handle, int(p), None, None, None, None, w.ctypes.data,
                                                  J.ctypes.data))
        out.update(weights=w[:nnz], objective=J)
    return out


class Plan2D:
    """Owner of an infft2d_plan_t handle (the 2-D tensor-product form)."""

    def __init__(self, handle, M1, M2, N, Ms1, Ms2, m):
        self.handle, self.M1, self.M2, self.N, self.m = handle, M1, M2, N, m
        self.M_sigma1, self.M_sigma2 = Ms1, Ms2

    def close(self):
        if self.handle:
            _check(library().infft2d_plan_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def infft2d_plan_create(M1, M2, N, sigma=2.0, m=4, kernel="full", tau=1e-12):
    h = ctypes.c_void_p()
    k = _KERNELS.get(kernel, kernel)
    _check(library().infft2d_plan_create(int(M1), int(M2), int(N), float(sigma), int(m), int(k), float(tau),
                                         ctypes.byref(h)))
    return Plan2D(h.value, int(M1), int(M2), int(N), int(round(sigma * M1)), int(round(sigma * M2)), int(m))


def infft2d_set_nodes(plan, x, stream=None):
    """x: (N, 2) float64 nodes (host or device); synchronous."""
    keep = []
    _check(library().infft2d_set_nodes(plan.handle, _as_ptr(x, "f64", keep), _stream(stream, x)))


def infft2d_precompute(plan, stream=None):
    _check(library().infft2d_precompute(plan.handle, _stream(stream)))


def _apply2(fn, plan, f, out, kind, stream):
    keep = []
    if out is None:
        out = _empty_like(f, plan.M1 * plan.M2, kind)
    _check(fn(plan.handle, _as_ptr(f, kind, keep), _as_ptr(out, kind, keep), _stream(stream, f, out)))
    return out.reshape(plan.M1, plan.M2)


def infft2d_apply(plan, f, out=None, stream=None):
    """fhat (M1 x M2 complex64, k1-major) = D^* F^* B_opt^* f for N complex64 samples."""
    return _apply2(library().infft2d_apply, plan, f, out, "c64", stream)


def infft2d_apply_z(plan, f, out=None, stream=None):
    return _apply2(library().infft2d_apply_z, plan, f, out, "c128", stream)


def infft2d_get_info(plan):
    info = _Info2D()
    _check(library().infft2d_get_info(plan.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in _Info2D._fields_}


def infft2d_copy_plan_data(plan, weights=True):
    """Pattern (col_offset, col_node) and, once precomputed, B_opt (weights, objective) as numpy arrays."""
    info = infft2d_get_info(plan)
    P = plan.M_sigma1 * plan.M_sigma2
    nnz = int(info["nnz"])
    off = np.empty(P + 1, np.int32)
    node = np.empty(max(nnz, 1), np.int32)
    w = np.empty(max(nnz, 1), np.float64) if weights else None
    J = np.empty(P, np.float64) if weights else None
    ptr = lambda a: a.ctypes.data if a is not None else None
    _check(library().infft2d_copy_plan_data(plan.handle, ptr(off), ptr(node), ptr(w), ptr(J)))
    out = dict(col_offset=off, col_node=node[:nnz])
    if weights:
        out.update(weights=w[:nnz], objective=J)
    return out
