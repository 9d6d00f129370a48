"""ctypes binding of the RS-S C ABI (``include/rss.h``), same names as the C calls.

Only argument marshalling happens here.  Device buffers are torch tensors
(``torch.float64`` or ``torch.complex128`` on CUDA); host buffers are numpy
arrays.  Right-hand sides are n x nrhs column-major: a tensor of shape
(n, nrhs) with stride (1, ldb), e.g. ``torch.empty(nrhs, n).T``, or a 1-D
tensor of length n.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

LAPLACE, HELMHOLTZ, TEST_POLY, TEST_RPOLY, HELMHOLTZ_LS = 0, 1, 2, 3, 4
MAX_COEF = 8
_STATUS = {0: "RSS_OK", 1: "RSS_EINVAL", 2: "RSS_ENOMEM", 3: "RSS_ECUDA", 4: "RSS_ENUMERIC",
           5: "RSS_ETIMEOUT", 6: "RSS_EBUSY"}

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "librss_gb300.so")


class RSSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("h", ctypes.c_double), ("kappa", ctypes.c_double),
                ("diag_re", ctypes.c_double), ("diag_im", ctypes.c_double),
                ("proxy_n", ctypes.c_int), ("proxy_radius_over_side", ctypes.c_double),
                ("eps", ctypes.c_double), ("ncoef", ctypes.c_int),
                ("coef_re", ctypes.c_double * MAX_COEF), ("coef_im", ctypes.c_double * MAX_COEF),
                ("scale", ctypes.c_double), ("phase_x", ctypes.c_double),
                ("phase_y", ctypes.c_double), ("id_rows", ctypes.c_int),
                ("schur_path", ctypes.c_int), ("id_cluster", ctypes.c_int),
                ("bump_cx", ctypes.c_double), ("bump_cy", ctypes.c_double),
                ("bump_a", ctypes.c_double), ("diag_rule", ctypes.c_int), ("per_box", ctypes.c_int),
                ("class_order", ctypes.c_int), ("wait_polls", ctypes.c_int),
                ("tune_table", ctypes.c_char_p)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"RS-S CUDA library not built: {path} is missing "
                          "(run python -m paper_2310_15458_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.rss_build_tree.argtypes = [vp, i64, ctypes.c_int, ctypes.POINTER(vp)]
    lib.rss_factor.argtypes = [vp, ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]
    lib.rss_solve.argtypes = [vp, vp, i64, i64, vp]
    lib.rss_solve_noalloc.argtypes = [vp, vp, i64, i64, vp]
    lib.rss_server_create.argtypes = [ctypes.c_size_t, i64, ctypes.POINTER(vp)]
    lib.rss_server_add.argtypes = [vp, vp, ctypes.POINTER(i32)]
    lib.rss_server_submit.argtypes = [vp, i32, vp, vp, i64, ctypes.POINTER(i64)]
    lib.rss_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.rss_server_stats.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.rss_free.argtypes = [vp]
    lib.rss_free.restype = None
    lib.rss_last_error.restype = ctypes.c_char_p
    lib.rss_info.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.rss_level_ranks.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i32)]
    lib.rss_box_record.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(i32)] + [vp] * 8
    dp = ctypes.POINTER(ctypes.c_double)
    lib.rss_self_integral.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
    lib.rss_matvec.argtypes = [vp, vp, vp, i64, i64, vp]
    lib.rss_solve_iterative.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, vp]
    lib.rss_trim_memory.argtypes = [ctypes.c_size_t]
    lib.rss_probe_fp64.argtypes = [dp, dp, vp]
    lib.rss_probe_dmma.argtypes = [dp, dp, vp]
    lib.rss_tune_solve.argtypes = [vp, i64, vp, ctypes.c_char_p, ctypes.c_size_t]
    for name in ("rss_build_tree", "rss_factor", "rss_solve", "rss_solve_noalloc", "rss_info",
                 "rss_level_ranks", "rss_box_record", "rss_server_create", "rss_server_add",
                 "rss_server_submit", "rss_server_wait", "rss_server_stats", "rss_self_integral",
                 "rss_matvec", "rss_solve_iterative", "rss_trim_memory", "rss_probe_fp64",
                 "rss_probe_dmma", "rss_tune_solve"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise RSSError(status, _load().rss_last_error().decode())


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream or None
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream) or None


class Tree:
    """Quadtree handle (rss_tree)."""

    def __init__(self, handle, n, side, leaf):
        self._h, self.n, self.side, self.leaf = handle, n, side, leaf

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rss_free(self._h)
            self._h = None


class Factor:
    """Factorization handle (rss_factorization)."""

    def __init__(self, handle, n, is_complex, tree):
        self._h, self.n, self.is_complex, self.tree = handle, n, is_complex, tree

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rss_free(self._h)
            self._h = None


def rss_build_tree(points: np.ndarray, leaf: int = 64) -> Tree:
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != 2:
        raise ValueError("points must have shape (n, 2)")
    h = ctypes.c_void_p()
    _check(lib.rss_build_tree(pts.ctypes.data, pts.shape[0], leaf, ctypes.byref(h)))
    side = int(round(np.sqrt(pts.shape[0])))
    return Tree(h, pts.shape[0], side, leaf)


def rss_factor(tree: Tree, kind: int = LAPLACE, eps: float = 1e-6, h: float = 0.0,
               kappa: float = 0.0, diag: complex = 1.0, proxy_n: int = 64,
               proxy_radius_over_side: float = 1.25, coef=(), scale: float = 1.0,
               phase=(0.0, 0.0), full_stack: bool = False, schur_fp64: bool = False,
               id_cluster: int = 0, diag_rule: int = 0, bump=(0.5, 0.5, 32.0),
               per_box: bool = False, schur_mma_sync: bool = False, class_order: int = 0,
               wait_polls: int = 0, tune_table: dict | str | None = None, stream=None) -> Factor:
    lib = _load()
    p = _Params()
    p.kind, p.h, p.kappa = kind, h, kappa
    p.diag_re, p.diag_im = complex(diag).real, complex(diag).imag
    p.proxy_n, p.proxy_radius_over_side, p.eps = proxy_n, proxy_radius_over_side, eps
    coef = list(coef)
    if len(coef) > MAX_COEF:
        raise ValueError("too many coefficients")
    p.ncoef = len(coef)
    for i, c in enumerate(coef):
        p.coef_re[i], p.coef_im[i] = complex(c).real, complex(c).imag
    p.scale, p.phase_x, p.phase_y = scale, phase[0], phase[1]
    p.id_rows = 1 if full_stack else 0
    p.schur_path = 1 if schur_fp64 else (2 if schur_mma_sync else 0)
    p.id_cluster = id_cluster
    p.bump_cx, p.bump_cy, p.bump_a = bump
    p.diag_rule = diag_rule
    p.per_box = 1 if per_box else 0
    p.class_order = int(class_order)
    p.wait_polls = int(wait_polls)
    if tune_table is not None:
        p.tune_table = (json.dumps(tune_table) if isinstance(tune_table, dict) else str(tune_table)).encode()
    out = ctypes.c_void_p()
    _check(lib.rss_factor(tree.handle, ctypes.byref(p), _stream_handle(stream), ctypes.byref(out)))
    return Factor(out, tree.n, kind in (HELMHOLTZ, TEST_POLY, HELMHOLTZ_LS), tree)


def rss_self_integral(kind: int, h: float, kappa: float = 0.0) -> complex:
    """Integral of the kernel over one h x h cell (Eqs. 16 and 20)."""
    lib = _load()
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib.rss_self_integral(kind, h, kappa, ctypes.byref(re), ctypes.byref(im)))
    return complex(re.value, im.value)


def _columns(t, n: int, name: str) -> tuple[int, int]:
    """(nrhs, ld) of an n x nrhs column-major tensor: shape (n,) or (n, nrhs) with
    stride (1, ld).  With more than one column, ld must be at least n, so that the
    columns do not overlap (an expanded tensor, whose columns share storage, is
    refused: the library would read and write n * nrhs entries through it)."""
    if t.dim() not in (1, 2):
        raise ValueError(f"{name} must be 1-D or 2-D")
    if t.shape[0] != n:
        raise ValueError(f"{name} has the wrong number of rows")
    if t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major: shape (n, nrhs), stride (1, ld)")
    if t.dim() == 1 or t.shape[1] == 1:
        return 1, n
    if t.stride(1) < n:
        raise ValueError(f"{name}: columns overlap (stride {t.stride(1)} < {n} rows)")
    return t.shape[1], t.stride(1)


def _dev_vector(f: Factor, t, name):
    import torch
    want = torch.complex128 if f.is_complex else torch.float64
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != want:
        raise TypeError(f"{name} must be a CUDA tensor of {want}")
    if t.shape[0] != f.n or t.stride(0) != 1:
        raise ValueError(f"{name} must have n rows, contiguous down the column")
    return t


def rss_matvec(f: Factor, x, y=None, stream=None):
    """y = A x by FFT (x: (n,) or (n, nrhs) column-major CUDA tensor); returns y."""
    import torch
    x = _dev_vector(f, x, "x")
    if y is None:
        y = torch.empty_like(x) if x.dim() == 1 else torch.empty(x.shape[1], x.shape[0], dtype=x.dtype,
                                                                  device=x.device).T
    y = _dev_vector(f, y, "y")
    nrhs, ld = _columns(x, f.n, "x")
    if _columns(y, f.n, "y") != (nrhs, ld):
        raise ValueError("x and y must have the same shape and leading dimension")
    _check(_load().rss_matvec(f.handle, x.data_ptr(), y.data_ptr(), nrhs, ld, _stream_handle(stream)))
    return y


def rss_solve_iterative(f: Factor, b, tol: float = 1e-12, maxit: int = 200, restart: int = 20,
                        method: int = 0, stream=None):
    """x with ||b - A x|| <= tol ||b||, the factorization as preconditioner (PCG or
    GMRES); returns (x, iterations, relative residual)."""
    import torch
    b = _dev_vector(f, b, "b")
    if b.dim() != 1:
        raise ValueError("b must be a single right-hand side")
    x = torch.empty_like(b)
    it, rel = ctypes.c_int(), ctypes.c_double()
    _check(_load().rss_solve_iterative(f.handle, b.data_ptr(), x.data_ptr(), tol, maxit, restart, method,
                                       ctypes.byref(it), ctypes.byref(rel), _stream_handle(stream)))
    return x, it.value, rel.value


def rss_solve(f: Factor, b, stream=None):
    """Overwrite b with A^{-1} b; returns b."""
    lib = _load()
    if isinstance(b, np.ndarray):
        want = np.complex128 if f.is_complex else np.float64
        if b.dtype != want:
            raise TypeError(f"b must be {want.__name__}")
        if not b.flags.writeable:
            raise ValueError("b must be writeable (it is overwritten by the solution)")
        if b.ndim == 1:
            nrhs, ldb = 1, b.shape[0]
            if not b.flags.c_contiguous:
                raise ValueError("b must be contiguous")
        else:
            if b.strides[0] != b.itemsize:
                raise ValueError("b must be column-major (Fortran order)")
            nrhs = b.shape[1]
            # a single column may carry any stride for its (unused) second axis
            ldb = b.shape[0] if nrhs == 1 else b.strides[1] // b.itemsize
            if nrhs > 1 and ldb < b.shape[0]:
                raise ValueError(f"b: columns overlap (stride {ldb} < {b.shape[0]} rows)")
        if b.shape[0] != f.n:
            raise ValueError("b has the wrong number of rows")
        _check(lib.rss_solve(f.handle, b.ctypes.data, nrhs, ldb, _stream_handle(stream)))
        return b
    import torch
    want = torch.complex128 if f.is_complex else torch.float64
    if b.dtype != want:
        raise TypeError(f"b must be {want}")
    nrhs, ldb = _columns(b, f.n, "b")
    _check(lib.rss_solve(f.handle, b.data_ptr(), nrhs, ldb, _stream_handle(stream)))
    return b


def rss_solve_noalloc(f: Factor, b, stream=None):
    """rss_solve for callers that cannot allocate device memory: b must be a CUDA
    tensor and n * nrhs scalars must fit the library's fixed 16 MiB scratch array,
    which every call shares (overlapping calls race).  Overwrites b; returns b."""
    import torch
    want = torch.complex128 if f.is_complex else torch.float64
    if not isinstance(b, torch.Tensor) or not b.is_cuda or b.dtype != want:
        raise TypeError(f"b must be a CUDA tensor of {want}")
    nrhs, ldb = _columns(b, f.n, "b")
    _check(_load().rss_solve_noalloc(f.handle, b.data_ptr(), nrhs, ldb, _stream_handle(stream)))
    return b


def rss_tune_solve(f: Factor, nrhs: int = 1, stream=None) -> dict:
    """Time the solve's launch schedules on f, keep the fastest for its later
    solves, and return the table (rss_params.tune_table accepts it back)."""
    buf = ctypes.create_string_buffer(4096)
    _check(_load().rss_tune_solve(f.handle, int(nrhs), _stream_handle(stream), buf, len(buf)))
    return json.loads(buf.value.decode())


def rss_probe_fp64(stream=None) -> tuple[float, float]:
    """Measured FP64 FMA throughput of the current device: (TFLOP/s, ms per launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(_load().rss_probe_fp64(ctypes.byref(t), ctypes.byref(ms), _stream_handle(stream)))
    return t.value, ms.value


def rss_probe_dmma(stream=None) -> tuple[float, float]:
    """Measured FP64 tensor-core (mma.sync f64) throughput: (TFLOP/s, ms per launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(_load().rss_probe_dmma(ctypes.byref(t), ctypes.byref(ms), _stream_handle(stream)))
    return t.value, ms.value


def rss_free(obj):
    if obj is not None and getattr(obj, "_h", None):
        _load().rss_free(obj._h)
        obj._h = None


def rss_trim_memory(keep_bytes: int = 0):
    """Return reserved but unused memory of the library's device pool to the
    driver, keeping at most ``keep_bytes`` reserved (waits for the device)."""
    _check(_load().rss_trim_memory(int(keep_bytes)))


def rss_info(f: Factor) -> dict:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_load().rss_info(f.handle, buf, len(buf)))
    return json.loads(buf.value.decode())


def rss_level_ranks(f: Factor, side: int) -> np.ndarray:
    out = np.zeros(side * side, dtype=np.int32)
    _check(_load().rss_level_ranks(f.handle, side, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return out


def rss_box_record(f: Factor, side: int, box: int) -> dict:
    """S, R, C (caller's point indices), T, LU, piv, E, F of one eliminated box."""
    lib = _load()
    sizes = np.zeros(4, dtype=np.int32)
    pi32 = ctypes.POINTER(ctypes.c_int32)
    _check(lib.rss_box_record(f.handle, side, box, sizes.ctypes.data_as(pi32), *([None] * 8)))
    k, r, c, n = (int(v) for v in sizes)
    dt = np.complex128 if f.is_complex else np.float64
    S, R, C = np.zeros(k, np.int64), np.zeros(r, np.int64), np.zeros(c, np.int64)
    T = np.zeros((k, r), dt, order="F")
    LU = np.zeros((r, r), dt, order="F")
    piv = np.zeros(r, np.int32)
    E = np.zeros((c, r), dt, order="F")
    F = np.zeros((r, c), dt, order="F")
    _check(lib.rss_box_record(f.handle, side, box, sizes.ctypes.data_as(pi32),
                              S.ctypes.data, R.ctypes.data, C.ctypes.data, T.ctypes.data,
                              LU.ctypes.data, piv.ctypes.data, E.ctypes.data, F.ctypes.data))
    return dict(k=k, r=r, c=c, n=n, S=S, R=R, C=C, T=T, LU=LU, piv=piv, E=E, F=F)


class Server:
    """Solve server handle (rss_server): resident factorizations, continuous batching."""

    def __init__(self, handle):
        self._h = handle
        self._factors = []      # keep registered factorizations alive
        self._held = {}         # ticket -> (b, x) buffers the worker reads and writes

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rss_free(self._h)
            self._h = None


def rss_server_create(device_bytes: int, max_batch_rhs: int = 256) -> Server:
    h = ctypes.c_void_p()
    _check(_load().rss_server_create(device_bytes, max_batch_rhs, ctypes.byref(h)))
    return Server(h)


def rss_server_add(s: Server, f: Factor) -> int:
    fid = ctypes.c_int32()
    _check(_load().rss_server_add(s.handle, f.handle, ctypes.byref(fid)))
    s._factors.append(f)
    return fid.value


def rss_server_submit(s: Server, factor_id: int, b: np.ndarray, x: np.ndarray | None = None) -> int:
    """Queue A^{-1} b; b is (n,) or (n, nrhs) Fortran-ordered.  Returns a ticket."""
    b = np.asfortranarray(b)
    if x is None:
        x = np.empty_like(b, order="F")
    nrhs = 1 if b.ndim == 1 else b.shape[1]
    t = ctypes.c_int64()
    _check(_load().rss_server_submit(s.handle, factor_id, b.ctypes.data, x.ctypes.data, nrhs,
                                     ctypes.byref(t)))
    s._held[t.value] = (b, x)
    return t.value


def rss_server_wait(s: Server, ticket: int, timeout: float = 0.0):
    """Wait for a ticket; returns (x, latency in seconds)."""
    lat = ctypes.c_double()
    try:
        _check(_load().rss_server_wait(s.handle, ticket, timeout, ctypes.byref(lat)))
    finally:
        pass
    b, x = s._held.pop(ticket)
    return x, lat.value


def rss_server_stats(s: Server) -> dict:
    buf = ctypes.create_string_buffer(4096)
    _check(_load().rss_server_stats(s.handle, buf, len(buf)))
    return json.loads(buf.value.decode())
