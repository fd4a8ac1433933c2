"""GB300 finite-temperature Lanczos (FTLM) for anisotropic spin Hamiltonians.

A thin ctypes binding of the C ABI in ``include/ftlm.h``: every function here
only marshals arguments; all work runs in ``libftlm_gb300.so`` (CUDA kernels
for sm_103a plus the host eigensolver).  There is no Python or CPU fallback:
if the library is missing, every call raises.

Device vector blocks are passed as raw device pointers (ints) or as objects
with ``data_ptr()`` (e.g. torch tensors of dtype complex64 / complex128 with
shape [dim, nvec], contiguous).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_LIB_PATH = _build.LIB

C128, C64 = 0, 1
START_RANDOM, START_BASIS, START_USER, START_PAIRS = 0, 1, 2, 3
_DTYPES = {"c128": C128, "complex128": C128, C128: C128, "c64": C64, "complex64": C64, C64: C64}
_STATUS = {0: "FTLM_OK", 1: "FTLM_ERR_INVALID_ARG", 2: "FTLM_ERR_OUT_OF_MEMORY", 3: "FTLM_ERR_CUDA",
           4: "FTLM_ERR_TIMEOUT", 5: "FTLM_ERR_UNSUPPORTED", 6: "FTLM_ERR_NUMERICAL"}


class FtlmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Constants(ctypes.Structure):
    _fields_ = [("mu_B", ctypes.c_double), ("C_dip", ctypes.c_double)]


class RunParams(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_int), ("M", ctypes.c_int), ("seed", ctypes.c_uint64), ("vec_offset", ctypes.c_uint64),
        ("dtype", ctypes.c_int), ("start", ctypes.c_int), ("basis_offset", ctypes.c_uint64),
        ("user_start", ctypes.c_void_p), ("T", ctypes.POINTER(ctypes.c_double)), ("nT", ctypes.c_int),
        ("obs_dir", ctypes.POINTER(ctypes.c_double)), ("breakdown_tol", ctypes.c_double),
        ("autotune", ctypes.c_int), ("time_kernels", ctypes.c_int), ("stream", ctypes.c_void_p),
        ("symmetric", ctypes.c_int), ("reorth", ctypes.c_int),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("lnZ", ctypes.POINTER(ctypes.c_double)), ("E", ctypes.POINTER(ctypes.c_double)),
        ("C", ctypes.POINTER(ctypes.c_double)), ("M_B", ctypes.POINTER(ctypes.c_double)),
        ("M_B_imag", ctypes.POINTER(ctypes.c_double)), ("alpha", ctypes.POINTER(ctypes.c_double)),
        ("beta", ctypes.POINTER(ctypes.c_double)), ("p", ctypes.POINTER(ctypes.c_double)),
        ("M_eff", ctypes.POINTER(ctypes.c_int)), ("E0", ctypes.c_double), ("device_ms", ctypes.c_double),
        ("hv_ms", ctypes.c_double), ("hv_launches", ctypes.c_int), ("kernel_launches", ctypes.c_int),
        ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
        ("cube_bits", ctypes.c_int), ("passes", ctypes.c_int), ("group_vectors", ctypes.c_int),
        ("tile_rows", ctypes.c_int),
        ("grid", ctypes.c_int), ("threads", ctypes.c_int), ("vector_major", ctypes.c_int),
        ("M_B_sym", ctypes.POINTER(ctypes.c_double)), ("M_B_sym_imag", ctypes.POINTER(ctypes.c_double)),
        ("O_lanczos", ctypes.POINTER(ctypes.c_double)), ("sym_ms", ctypes.c_double),
        ("gap_ms", ctypes.c_double), ("site_cube", ctypes.c_int),
    ]


# every symbol include/ftlm.h declares
EXPORTS = ["ftlm_system_create", "ftlm_system_destroy", "ftlm_system_dim", "ftlm_system_table_bytes",
           "ftlm_apply_h", "ftlm_apply_sdir",
           "ftlm_start_block", "ftlm_start_block_noalloc", "ftlm_start_pairs", "ftlm_time_reverse",
           "ftlm_run", "ftlm_run_batch", "ftlm_sums", "ftlm_sums_sym",
           "ftlm_csr_create", "ftlm_csr_nnz", "ftlm_csr_bytes", "ftlm_csr_apply", "ftlm_csr_destroy",
           "ftlm_tune_shape", "ftlm_last_error", "ftlm_version"]

_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library (nvcc, sm_103a) in-tree."""
    return _build.build(force=force)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"CUDA library {_LIB_PATH} is missing: run paper_2607_25585_gb300.build()")
        L = ctypes.CDLL(_LIB_PATH)
        P, vp, d, i = ctypes.POINTER, ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        pd = P(d)
        L.ftlm_system_create.argtypes = [i, P(i), pd, pd, pd, d, pd, pd, P(Constants), P(vp)]
        L.ftlm_system_destroy.argtypes = [vp]
        L.ftlm_system_destroy.restype = None
        L.ftlm_system_dim.argtypes = [vp]
        L.ftlm_system_dim.restype = ctypes.c_uint64
        L.ftlm_system_table_bytes.argtypes = [vp]
        L.ftlm_system_table_bytes.restype = ctypes.c_uint64
        L.ftlm_apply_h.argtypes = [vp, vp, vp, i, i, vp]
        L.ftlm_apply_sdir.argtypes = [vp, pd, vp, vp, i, i, vp]
        L.ftlm_start_block.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, vp, i, i, vp]
        L.ftlm_start_block_noalloc.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, vp, i, i, vp]
        L.ftlm_start_pairs.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, vp, i, i, vp]
        L.ftlm_time_reverse.argtypes = [vp, vp, vp, i, i, vp]
        L.ftlm_run.argtypes = [vp, P(RunParams), P(Result)]
        L.ftlm_run_batch.argtypes = [i, P(vp), P(RunParams), P(Result)]
        L.ftlm_sums.argtypes = [i, i, P(i), pd, pd, pd, d, d, pd, i, P(Result)]
        L.ftlm_sums_sym.argtypes = [i, i, P(i), pd, pd, pd, d, pd, i, pd, pd]
        L.ftlm_csr_create.argtypes = [vp, i, P(vp)]
        L.ftlm_csr_nnz.restype = ctypes.c_uint64
        L.ftlm_csr_nnz.argtypes = [vp]
        L.ftlm_csr_bytes.restype = ctypes.c_uint64
        L.ftlm_csr_bytes.argtypes = [vp]
        L.ftlm_csr_apply.argtypes = [vp, vp, vp, i, vp]
        L.ftlm_csr_destroy.argtypes = [vp]
        L.ftlm_csr_destroy.restype = None
        L.ftlm_tune_shape.argtypes = [vp, i, i, i, i, i, i]
        L.ftlm_last_error.restype = ctypes.c_char_p
        L.ftlm_version.restype = ctypes.c_char_p
        for f in ("ftlm_system_create", "ftlm_apply_h", "ftlm_apply_sdir", "ftlm_start_block", "ftlm_run",
                  "ftlm_run_batch", "ftlm_sums", "ftlm_tune_shape", "ftlm_start_block_noalloc"):
            getattr(L, f).restype = i
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise FtlmError(status, lib().ftlm_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s, *blocks):
    """cudaStream_t for a call: the given stream, else torch's current stream
    when device blocks are torch tensors (so the call is ordered with the
    tensors' producers and consumers), else the default stream."""
    if s is None:
        if any(hasattr(b, "data_ptr") for b in blocks):
            import torch
            return int(torch.cuda.current_stream().cuda_stream) or None
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


_ELEMENT_BYTES = {C128: 16, C64: 8}


def _check_block(t, dim: int, nvec: int, dtype, name="block"):
    """Checks a device block before its pointer goes to the library: for a
    tensor (an object with ``data_ptr()``), that it is on a CUDA device,
    contiguous, of the element size of ``dtype`` and holds at least
    dim * nvec elements; a raw pointer (int) is the caller's responsibility.
    Raises FtlmError(FTLM_ERR_INVALID_ARG) without calling the library."""
    if t is None or isinstance(t, int):
        return
    code = _DTYPES.get(dtype)
    if code is None:
        raise FtlmError(1, f"{name}: unknown dtype {dtype!r}")
    dev = getattr(t, "device", None)
    if dev is not None and getattr(dev, "type", "cuda") != "cuda":
        raise FtlmError(1, f"{name}: a device block is needed, got a tensor on {dev}")
    if hasattr(t, "is_contiguous") and not t.is_contiguous():
        raise FtlmError(1, f"{name}: the block must be contiguous")
    esz = t.element_size() if hasattr(t, "element_size") else None
    if esz is not None and esz != _ELEMENT_BYTES[code]:
        raise FtlmError(1, f"{name}: elements of {esz} bytes do not match dtype {dtype!r} "
                           f"({_ELEMENT_BYTES[code]} bytes)")
    n = t.numel() if hasattr(t, "numel") else None
    if n is not None and n < int(dim) * int(nvec):
        raise FtlmError(1, f"{name}: {n} elements, {int(dim) * int(nvec)} needed ([{dim}][{nvec}])")


def _check_device(sys, *blocks):
    """The tensors must live on the current CUDA device (the one the library
    enqueues on); raises FtlmError otherwise."""
    for t in blocks:
        dev = getattr(t, "device", None)
        if dev is None or getattr(dev, "index", None) is None:
            continue
        import torch
        if dev.index != torch.cuda.current_device():
            raise FtlmError(1, f"block on {dev}, current device is cuda:{torch.cuda.current_device()}")


def _pd(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


class System:
    """The spin Hamiltonian of Eq. (3) on the GPU (``ftlm_system_create``)."""

    def __init__(self, two_s, J=None, d_ion=None, e_axes=None, g=2.0, B=(0.0, 0.0, 0.0), pos=None,
                 mu_B=None, C_dip=None, name=None):
        L = lib()
        self.two_s = np.ascontiguousarray(two_s, dtype=np.int32)
        n = len(self.two_s)
        self.n = n
        self.g = float(g)
        self.name = name
        J = None if J is None else _f64(np.broadcast_to(J, (n, n)))
        d_ion = _f64(d_ion)
        e_axes = _f64(e_axes)
        pos = _f64(pos)
        B = _f64(B)
        k = None
        if mu_B is not None or C_dip is not None:
            k = Constants(0.6717 if mu_B is None else mu_B, 0.6228 if C_dip is None else C_dip)
        h = ctypes.c_void_p()
        _check(L.ftlm_system_create(n, self.two_s.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _pd(J), _pd(d_ion),
                                    _pd(e_axes), self.g, _pd(B), _pd(pos), ctypes.byref(k) if k else None,
                                    ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_dict(cls, w):
        return cls(w["two_s"], w["J"], w.get("d_ion"), w.get("e_axes"), w.get("g", 2.0), w["B"], w.get("pos"),
                   name=w.get("name"))

    @property
    def handle(self):
        return self._h

    @property
    def dim(self) -> int:
        return int(lib().ftlm_system_dim(self._h))

    @property
    def table_bytes(self) -> int:
        return int(lib().ftlm_system_table_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ftlm_system_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _blocks(sys, nvec, dtype, **blocks):
    for name, t in blocks.items():
        _check_block(t, sys.dim, nvec, dtype, name)
    _check_device(sys, *blocks.values())


def apply_h(sys: System, x, y, nvec: int, dtype="c64", stream=None):
    """y = H x on device blocks [dim][nvec] (``ftlm_apply_h``)."""
    _blocks(sys, nvec, dtype, x=x, y=y)
    _check(lib().ftlm_apply_h(sys.handle, _ptr(x), _ptr(y), int(nvec), _DTYPES[dtype], _stream(stream, x, y)))


def apply_sdir(sys: System, x, y, nvec: int, dtype="c64", u=None, stream=None):
    """y = (u.S) x (``ftlm_apply_sdir``); u = None uses the field direction."""
    _blocks(sys, nvec, dtype, x=x, y=y)
    uu = _f64(u)
    _check(lib().ftlm_apply_sdir(sys.handle, _pd(uu), _ptr(x), _ptr(y), int(nvec), _DTYPES[dtype],
                                 _stream(stream, x, y)))


def start_block(sys: System, out, nvec: int, seed: int, vec_offset: int = 0, dtype="c64", stream=None):
    """Normalised Gaussian start vectors into a device block (``ftlm_start_block``)."""
    _blocks(sys, nvec, dtype, out=out)
    _check(lib().ftlm_start_block(sys.handle, int(seed), int(vec_offset), _ptr(out), int(nvec), _DTYPES[dtype],
                                  _stream(stream, out)))


def start_pairs(sys: System, out, nvec: int, seed: int, vec_offset: int = 0, dtype="c64", stream=None):
    """Normalised pairs of time-reversed random vectors (``ftlm_start_pairs``)."""
    _blocks(sys, nvec, dtype, out=out)
    _check(lib().ftlm_start_pairs(sys.handle, int(seed), int(vec_offset), _ptr(out), int(nvec), _DTYPES[dtype],
                                  _stream(stream, out)))


def time_reverse(sys: System, x, y, nvec: int, dtype="c64", stream=None):
    """y = Theta x, Theta = exp(-i pi S^y) K (``ftlm_time_reverse``)."""
    _blocks(sys, nvec, dtype, x=x, y=y)
    _check(lib().ftlm_time_reverse(sys.handle, _ptr(x), _ptr(y), int(nvec), _DTYPES[dtype], _stream(stream, x)))


def start_block_noalloc(sys: System, out, nvec: int, seed: int, vec_offset: int = 0, dtype="c64", stream=None):
    """``ftlm_start_block`` without any device allocation, for callers that
    may not allocate (``ftlm_start_block_noalloc``): its scratch is a static
    device array inside the library, so at most 64 vectors, and calls that
    overlap on the GPU race on that array."""
    _blocks(sys, nvec, dtype, out=out)
    _check(lib().ftlm_start_block_noalloc(sys.handle, int(seed), int(vec_offset), _ptr(out), int(nvec),
                                          _DTYPES[dtype], _stream(stream, out)))


def _params(R, M, T, seed, vec_offset, dtype, start, basis_offset, user_start, obs_dir, breakdown_tol, autotune,
            time_kernels, stream, keep, symmetric=False, reorth=False):
    T = _f64(T)
    od = _f64(obs_dir)
    keep += [T, od]
    mode = {"random": START_RANDOM, "basis": START_BASIS, "user": START_USER, "pairs": START_PAIRS}[start] \
        if isinstance(start, str) \
        else int(start)
    return RunParams(int(R), int(M), int(seed), int(vec_offset), _DTYPES[dtype], mode, int(basis_offset),
                     _ptr(user_start), _pd(T), len(T), _pd(od), float(breakdown_tol), int(autotune),
                     int(time_kernels), _stream(stream, user_start), int(bool(symmetric)), int(bool(reorth)))


def _result(R, M, nT, keep, symmetric=False):
    out = {k: np.zeros(nT) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")}
    out.update(alpha=np.zeros((R, M)), beta=np.zeros((R, M)), p=np.zeros((R, M), dtype=np.complex128),
               M_eff=np.zeros(R, dtype=np.int32))
    if symmetric:
        out.update(M_B_sym=np.zeros(nT), M_B_sym_imag=np.zeros(nT), O=np.zeros((R, M, M), dtype=np.complex128))
    keep.append(out)
    r = Result(*[_pd(out[k]) for k in ("lnZ", "E", "C", "M_B", "M_B_imag", "alpha", "beta")],
               _pd(out["p"].view(np.float64)), out["M_eff"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if symmetric:
        r.M_B_sym = _pd(out["M_B_sym"])
        r.M_B_sym_imag = _pd(out["M_B_sym_imag"])
        r.O_lanczos = _pd(out["O"].view(np.float64))
    return r, out


def _finish(r, out):
    out.update(E0=r.E0, device_ms=r.device_ms, hv_ms=r.hv_ms, gap_ms=r.gap_ms, hv_launches=r.hv_launches,
               kernel_launches=r.kernel_launches, h2d_bytes=int(r.h2d_bytes), d2h_bytes=int(r.d2h_bytes),
               shape={"cube_bits": r.cube_bits, "passes": r.passes, "group_vectors": r.group_vectors,
                      "tile_rows": r.tile_rows,
                      "grid": r.grid, "threads": r.threads, "vector_major": r.vector_major,
                      "site_cube": r.site_cube})
    if "M_B_sym" in out:
        out["sym_ms"] = r.sym_ms
    return out


def run(sys: System, R: int, M: int, T, seed: int = 0, vec_offset: int = 0, dtype="c64", start="random",
        basis_offset: int = 0, user_start=None, obs_dir=None, breakdown_tol: float = 0.0, autotune=False,
        time_kernels=False, stream=None, symmetric=False, reorth=False) -> dict:
    """FTLM (``ftlm_run``): returns lnZ, E, C, M_B, M_B_imag per T, E0, and the
    per-vector alpha, beta, p, M_eff; with symmetric=True also the symmetric
    estimator M_B_sym, M_B_sym_imag (Eqs. E-2-G, E-2-H), the matrices
    O[r, i, j] = <v_i|u.S|v_j> and sym_ms; reorth=True re-orthogonalises every
    new Lanczos vector against all previous ones of its chain."""
    keep = []
    if user_start is not None:
        _check_block(user_start, sys.dim, R, dtype, "user_start")
    p = _params(R, M, T, seed, vec_offset, dtype, start, basis_offset, user_start, obs_dir, breakdown_tol, autotune,
                time_kernels, stream, keep, symmetric, reorth)
    r, out = _result(R, M, p.nT, keep, symmetric)
    _check(lib().ftlm_run(sys.handle, ctypes.byref(p), ctypes.byref(r)))
    return _finish(r, out)


def run_batch(systems, R: int, M: int, T, seed: int = 0, vec_offset: int = 0, dtype="c64", obs_dir=None,
              breakdown_tol: float = 0.0, autotune=False, time_kernels=False, stream=None, start="random",
              reorth=False) -> list:
    """FTLM for several systems in one graph (``ftlm_run_batch``); start is
    "random", "pairs" or "basis" (reorth=True is rejected: one system only)."""
    keep = []
    p = _params(R, M, T, seed, vec_offset, dtype, start, 0, None, obs_dir, breakdown_tol, autotune, time_kernels,
                stream, keep, reorth=reorth)
    n = len(systems)
    rs, outs = [], []
    for _ in range(n):
        r, o = _result(R, M, p.nT, keep)
        rs.append(r)
        outs.append(o)
    arr = (Result * n)(*rs)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in systems])
    _check(lib().ftlm_run_batch(n, hs, ctypes.byref(p), arr))
    return [_finish(arr[k], outs[k]) for k in range(n)]


def sums(alpha, beta, p, M_eff, dim, g, T) -> dict:
    """Eqs. (4)-(5) from gathered tridiagonal data (``ftlm_sums``, host only)."""
    a = _f64(alpha)
    R, M = a.shape
    b = _f64(beta)
    pc = np.ascontiguousarray(p, dtype=np.complex128)
    me = np.ascontiguousarray(M_eff, dtype=np.int32)
    T = _f64(T)
    keep = []
    out = {k: np.zeros(len(T)) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")}
    r = Result(*[_pd(out[k]) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")], None, None, None, None)
    keep.append(out)
    _check(lib().ftlm_sums(R, M, me.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _pd(a), _pd(b),
                           _pd(pc.view(np.float64)), float(dim), float(g), _pd(T), len(T), ctypes.byref(r)))
    out["E0"] = r.E0
    return out


class CsrMatrix:
    """H assembled as a stored sparse matrix on the device (``ftlm_csr_*``): the
    comparison path for the matrix-free ``apply_h``."""

    def __init__(self, sys: System, dtype="c64"):
        h = ctypes.c_void_p()
        _check(lib().ftlm_csr_create(sys.handle, _DTYPES[dtype], ctypes.byref(h)))
        self.handle = h.value
        self.dtype = dtype
        self.dim = sys.dim
        self.nnz = int(lib().ftlm_csr_nnz(self.handle))
        self.bytes = int(lib().ftlm_csr_bytes(self.handle))

    def apply(self, x, y, nvec: int, stream=None):
        for name, t in (("x", x), ("y", y)):
            _check_block(t, self.dim, nvec, self.dtype, name)
        _check(lib().ftlm_csr_apply(self.handle, _ptr(x), _ptr(y), int(nvec), _stream(stream, x)))

    def close(self):
        if getattr(self, "handle", None):
            lib().ftlm_csr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sums_sym(alpha, beta, O, M_eff, g, T):
    """Host-only symmetric estimator from per-vector data (``ftlm_sums_sym``):
    returns (M_B_sym, M_B_sym_imag)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    R, M = a.shape
    b = np.ascontiguousarray(beta, dtype=np.float64)
    Oc = np.ascontiguousarray(O, dtype=np.complex128)
    me = np.ascontiguousarray(M_eff, dtype=np.int32)
    T = _f64(T)
    mb, mbi = np.zeros(len(T)), np.zeros(len(T))
    _check(lib().ftlm_sums_sym(R, M, me.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _pd(a), _pd(b),
                               _pd(Oc.view(np.float64)), float(g), _pd(T), len(T), _pd(mb), _pd(mbi)))
    return mb, mbi


def tune_shape(sys: System, nvec: int, dtype="c64", cube_bits: int = 0, group_vectors: int = 1,
               tile_cubes: int = 2, multipass: int = 0):
    """Override the launch shape for (system shape, nvec, dtype) (``ftlm_tune_shape``).

    cube_bits = -1 drops the override; cube_bits = 0 selects the general
    kernel: on the row-major block (multipass 0) or, in runs, on the
    vector-major block (multipass 1: group_vectors = the register cube's
    group size, 4 or 8, or 0 for one row a thread; tile_cubes x 256 rows or
    bases per tile); cube_bits 2..4 select the spin-1/2 register-cube shapes."""
    _check(lib().ftlm_tune_shape(sys.handle, int(nvec), _DTYPES[dtype], int(cube_bits), int(group_vectors),
                                 int(tile_cubes), int(multipass)))


def version() -> str:
    return lib().ftlm_version().decode()
