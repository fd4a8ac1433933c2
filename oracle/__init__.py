"""CPU FP64 oracle for the FTLM hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
the two share no code (the seeded input generators in ``ftlm_workloads`` hold
none of the method's arithmetic).

Two independent oracles live here:

* ``ftlm_oracle.cpp`` (this wrapper): the algorithm step by step -- the
  Hamiltonian of Eq. (3) applied by column scatter in ladder form, Philox
  Gaussian start vectors (Eq. 2), the Lanczos recurrence (Sec. II.C), a cyclic
  Jacobi tridiagonal eigensolver and the FTLM sums of Eqs. (4)-(5).
* ``oracle.dense``: the plain definition -- H assembled from Kronecker
  products of spin matrices exactly as Eq. (3) is written, and exact
  diagonalisation, for d up to a few thousand.

Pins that tie these to something other than themselves live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftlm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_ftlm.so")

MU_B_DEFAULT = 0.6717   # K/T
C_DIP_DEFAULT = 0.6228  # K Angstrom^3 (mu0 mu_B^2 / 4 pi / k_B)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain C++17, OpenMP over random vectors)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _CSystem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("two_s", ctypes.POINTER(ctypes.c_int)),
        ("J", ctypes.POINTER(ctypes.c_double)),
        ("d_ion", ctypes.POINTER(ctypes.c_double)),
        ("e_axes", ctypes.POINTER(ctypes.c_double)),
        ("g", ctypes.c_double),
        ("B", ctypes.POINTER(ctypes.c_double)),
        ("pos", ctypes.POINTER(ctypes.c_double)),
        ("mu_B", ctypes.c_double),
        ("C_dip", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i64, i32, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        pd = P(d)
        _lib.oracle_dim.restype = i64
        _lib.oracle_dim.argtypes = [P(_CSystem)]
        _lib.oracle_pair_tensor.argtypes = [P(_CSystem), i32, i32, pd]
        _lib.oracle_apply_h.argtypes = [P(_CSystem), pd, pd, i64]
        _lib.oracle_apply_sdir.argtypes = [P(_CSystem), pd, pd, pd, i64]
        _lib.oracle_time_reverse.argtypes = [P(_CSystem), pd, pd, i64]
        _lib.oracle_sftlm_sums.argtypes = [i32, i32, P(i32), pd, pd, pd, d, pd, i32, pd, pd]
        _lib.oracle_sftlm.argtypes = [P(_CSystem), i32, i32, u64, u64, i32, i64, pd, i32, d, pd, pd, i32,
                                      pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, P(i32)]
        _lib.oracle_h_column.restype = i64
        _lib.oracle_h_column.argtypes = [P(_CSystem), i64, P(i64), pd, i64]
        _lib.oracle_philox4x32_10.argtypes = [P(ctypes.c_uint32)] * 3
        _lib.oracle_philox4x32_10.restype = None
        _lib.oracle_start_vectors.argtypes = [i64, i64, u64, u64, pd]
        _lib.oracle_lanczos.argtypes = [P(_CSystem), pd, i32, i32, d, pd, pd, pd, pd]
        _lib.oracle_tridiag_eig.argtypes = [i32, pd, pd, pd, pd]
        _lib.oracle_ftlm_sums.argtypes = [i32, i32, P(i32), pd, pd, pd, d, d, pd, i32,
                                          pd, pd, pd, pd, pd, pd]
        _lib.oracle_ftlm.argtypes = [P(_CSystem), i32, i32, u64, u64, i32, i64, pd, i32, d, pd,
                                     pd, i32, pd, pd, pd, pd, pd, pd, pd, pd, pd, P(i32)]
        _lib.oracle_ftlm_tridiag.argtypes = [P(_CSystem), i32, i32, u64, u64, i32, i64, pd, i32, d, pd,
                                             pd, pd, pd, P(i32)]
        _lib.oracle_num_threads.restype = i32
    return _lib


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


@dataclass
class System:
    """Raw system description (the inputs of Eq. 3), kept as numpy arrays."""

    two_s: np.ndarray
    J: np.ndarray
    g: float = 2.0
    B: np.ndarray = field(default_factory=lambda: np.zeros(3))
    d_ion: np.ndarray | None = None
    e_axes: np.ndarray | None = None
    pos: np.ndarray | None = None
    mu_B: float = MU_B_DEFAULT
    C_dip: float = C_DIP_DEFAULT

    def __post_init__(self):
        self.two_s = np.ascontiguousarray(self.two_s, dtype=np.int32)
        n = len(self.two_s)
        self.J = np.ascontiguousarray(np.broadcast_to(self.J, (n, n)), dtype=np.float64)
        self.B = np.ascontiguousarray(self.B, dtype=np.float64).reshape(3)
        if self.d_ion is not None:
            self.d_ion = np.ascontiguousarray(self.d_ion, dtype=np.float64).reshape(n)
        if self.e_axes is not None:
            self.e_axes = np.ascontiguousarray(self.e_axes, dtype=np.float64).reshape(n, 3)
        if self.pos is not None:
            self.pos = np.ascontiguousarray(self.pos, dtype=np.float64).reshape(n, 3)

    @property
    def n(self) -> int:
        return len(self.two_s)

    @property
    def dim(self) -> int:
        return int(np.prod(self.two_s.astype(np.int64) + 1))

    def c(self) -> _CSystem:
        s = _CSystem()
        s.n = self.n
        s.two_s = self.two_s.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        s.J = _pd(self.J)
        s.d_ion = _pd(self.d_ion)
        s.e_axes = _pd(self.e_axes)
        s.g = self.g
        s.B = _pd(self.B)
        s.pos = _pd(self.pos)
        s.mu_B = self.mu_B
        s.C_dip = self.C_dip
        self._keep = s  # arrays referenced by s stay alive through self
        return s


def _cx(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


def apply_h(sys: System, x: np.ndarray) -> np.ndarray:
    """y = H x for a block x of shape [d] or [d][nvec] (column scatter, FP64)."""
    lib = _load()
    vec = x.ndim == 1
    X = _cx(x).reshape(sys.dim, -1)
    Y = np.empty_like(X)
    cs = sys.c()
    rc = lib.oracle_apply_h(ctypes.byref(cs), _pd(X.view(np.float64)), _pd(Y.view(np.float64)), X.shape[1])
    assert rc == 0, "oracle_apply_h failed"
    return Y[:, 0] if vec else Y


def apply_sdir(sys: System, direction, x: np.ndarray) -> np.ndarray:
    """y = (u . S) x with S = sum_i s_i."""
    lib = _load()
    vec = x.ndim == 1
    X = _cx(x).reshape(sys.dim, -1)
    Y = np.empty_like(X)
    u = np.ascontiguousarray(direction, dtype=np.float64)
    cs = sys.c()
    rc = lib.oracle_apply_sdir(ctypes.byref(cs), _pd(u), _pd(X.view(np.float64)), _pd(Y.view(np.float64)),
                               X.shape[1])
    assert rc == 0
    return Y[:, 0] if vec else Y


def h_column(sys: System, nu: int):
    """Column nu of H (rows, complex values), duplicates merged."""
    lib = _load()
    cap = 64 * sys.n * sys.n + 64 * sys.n + 16
    rows = np.empty(cap, dtype=np.int64)
    vals = np.empty(2 * cap, dtype=np.float64)
    cs = sys.c()
    k = lib.oracle_h_column(ctypes.byref(cs), int(nu), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _pd(vals), cap)
    assert k >= 0
    return rows[:k].copy(), vals[: 2 * k].view(np.complex128).copy()


def h_rows(sys: System, rows, x: np.ndarray) -> np.ndarray:
    """(H x)[mu] for the listed rows, from columns of H and Hermiticity
    (H[mu][nu] = conj(H[nu][mu])): y_mu = sum_nu conj(H[nu][mu]) x_nu."""
    X = _cx(x).reshape(sys.dim, -1)
    out = np.empty((len(rows), X.shape[1]), dtype=np.complex128)
    for k, mu in enumerate(rows):
        r, v = h_column(sys, int(mu))
        out[k] = (np.conj(v)[:, None] * X[r]).sum(axis=0)
    return out


def pair_tensor(sys: System, i: int, j: int) -> np.ndarray:
    lib = _load()
    out = np.empty(9)
    cs = sys.c()
    assert lib.oracle_pair_tensor(ctypes.byref(cs), i, j, _pd(out)) == 0
    return out.reshape(3, 3)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, dtype=np.uint32)
    P = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_philox4x32_10(c.ctypes.data_as(P), k.ctypes.data_as(P), o.ctypes.data_as(P))
    return o


def start_vectors(d: int, R: int, seed: int, vec_offset: int = 0) -> np.ndarray:
    """[d][R] block: column k is random vector number vec_offset + k, normalised."""
    lib = _load()
    out = np.empty((d, R), dtype=np.complex128)
    assert lib.oracle_start_vectors(d, R, seed, vec_offset, _pd(out.view(np.float64))) == 0
    return out


def time_reverse(sys: System, x: np.ndarray) -> np.ndarray:
    """Theta x = exp(-i pi S^y) K x for a [d] or [d][R] block (Sec. II.B)."""
    lib = _load()
    xx = _cx(x)
    shape = xx.shape
    xx = xx.reshape(sys.dim, -1)
    y = np.empty_like(xx)
    cs = sys.c()
    assert lib.oracle_time_reverse(ctypes.byref(cs), _pd(xx.view(np.float64)), _pd(y.view(np.float64)),
                                   xx.shape[1]) == 0
    return y.reshape(shape)


def start_pairs(sys: System, R: int, seed: int, vec_offset: int = 0) -> np.ndarray:
    """[d][R] block of time-reversed pairs: global vector v = vec_offset + k is
    random vector v // 2 (normalised), time-reversed when v is odd."""
    base = start_vectors(sys.dim, (vec_offset + R + 1) // 2 - vec_offset // 2, seed, vec_offset // 2)
    out = np.empty((sys.dim, R), dtype=np.complex128)
    for k in range(R):
        v = vec_offset + k
        col = base[:, v // 2 - vec_offset // 2]
        out[:, k] = time_reverse(sys, col) if v % 2 else col
    return out


def lanczos(sys: System, v0: np.ndarray, M: int, reorth: bool = False, tol: float = 1e-12, direction=None):
    """One Lanczos run; returns (alpha, beta, p, M_eff)."""
    lib = _load()
    v = _cx(v0).reshape(sys.dim)
    a = np.zeros(M)
    b = np.zeros(M)
    p = np.zeros(M, dtype=np.complex128)
    u = None if direction is None else np.ascontiguousarray(direction, dtype=np.float64)
    cs = sys.c()
    m = lib.oracle_lanczos(ctypes.byref(cs), _pd(v.view(np.float64)), M, int(reorth), tol, _pd(u), _pd(a),
                           _pd(b), _pd(p.view(np.float64)))
    assert m > 0
    return a, b, p, m


def tridiag_eig(alpha, beta):
    """Cyclic-Jacobi eigenpairs of tridiag(alpha, beta); U[k, n] = U_kn."""
    lib = _load()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    m = len(a)
    b = np.zeros(m)
    b[: m - 1] = np.asarray(beta, dtype=np.float64)[: m - 1]
    ev = np.empty(m)
    U = np.empty((m, m))
    assert lib.oracle_tridiag_eig(m, _pd(a), _pd(b), _pd(ev), _pd(U)) == 0
    return ev, U


def default_temperatures(nT: int = 40, Tmin: float = 0.05, Tmax: float = 50.0) -> np.ndarray:
    return Tmin * (Tmax / Tmin) ** (np.arange(nT) / (nT - 1))


def ftlm_sums(alpha, beta, p, M_eff, dim, g, T):
    """Eqs. (4)-(5) from per-run tridiagonal data [R][M]."""
    lib = _load()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    R, M = a.shape
    b = np.ascontiguousarray(beta, dtype=np.float64)
    pc = _cx(p)
    me = np.ascontiguousarray(M_eff, dtype=np.int32)
    T = np.ascontiguousarray(T, dtype=np.float64)
    nT = len(T)
    out = {k: np.empty(nT) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")}
    E0 = np.zeros(1)
    rc = lib.oracle_ftlm_sums(R, M, me.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _pd(a), _pd(b),
                              _pd(pc.view(np.float64)), float(dim), float(g), _pd(T), nT,
                              *[_pd(out[k]) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")], _pd(E0))
    assert rc == 0
    out["E0"] = float(E0[0])
    return out


def ftlm(sys: System, R: int, M: int, T=None, seed: int = 0, vec_offset: int = 0, start: str = "random",
         basis_offset: int = 0, user_start=None, reorth: bool = False, tol: float = 1e-12, direction=None):
    """Full FTLM run; returns a dict with lnZ, E, C, M_B, M_B_imag, E0,
    alpha, beta, p, M_eff."""
    lib = _load()
    T = default_temperatures() if T is None else np.ascontiguousarray(T, dtype=np.float64)
    nT = len(T)
    mode = {"random": 0, "basis": 1, "user": 2, "pairs": 3}[start]
    us = None
    if mode == 2:
        us = _cx(user_start).reshape(sys.dim, R)
    out = {k: np.empty(nT) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")}
    E0 = np.zeros(1)
    a = np.zeros((R, M))
    b = np.zeros((R, M))
    p = np.zeros((R, M), dtype=np.complex128)
    me = np.zeros(R, dtype=np.int32)
    u = None if direction is None else np.ascontiguousarray(direction, dtype=np.float64)
    cs = sys.c()
    rc = lib.oracle_ftlm(ctypes.byref(cs), R, M, seed, vec_offset, mode, basis_offset,
                         _pd(us.view(np.float64)) if us is not None else None, int(reorth), tol, _pd(u), _pd(T),
                         nT, *[_pd(out[k]) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")], _pd(E0), _pd(a), _pd(b),
                         _pd(p.view(np.float64)), me.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert rc == 0, "oracle_ftlm failed"
    out.update(E0=float(E0[0]), alpha=a, beta=b, p=p, M_eff=me, T=T)
    return out


def ftlm_tridiag(sys: System, R: int, M: int, seed: int = 0, vec_offset: int = 0, start: str = "random",
                 basis_offset: int = 0, reorth: bool = False, tol: float = 1e-12, direction=None):
    """The Lanczos half of ``ftlm`` alone (R recurrences, one host thread
    each): alpha, beta, p [R][M] and M_eff [R], no eigensolve or sums."""
    lib = _load()
    mode = {"random": 0, "basis": 1, "pairs": 3}[start]
    a = np.zeros((R, M))
    b = np.zeros((R, M))
    p = np.zeros((R, M), dtype=np.complex128)
    me = np.zeros(R, dtype=np.int32)
    u = None if direction is None else np.ascontiguousarray(direction, dtype=np.float64)
    cs = sys.c()
    rc = lib.oracle_ftlm_tridiag(ctypes.byref(cs), R, M, seed, vec_offset, mode, basis_offset, None, int(reorth), tol,
                                 _pd(u), _pd(a), _pd(b), _pd(p.view(np.float64)),
                                 me.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert rc == 0, "oracle_ftlm_tridiag failed"
    return {"alpha": a, "beta": b, "p": p, "M_eff": me}


def sftlm(sys: System, R: int, M: int, T=None, seed: int = 0, vec_offset: int = 0, start: str = "random",
          basis_offset: int = 0, user_start=None, reorth: bool = False, tol: float = 1e-12, direction=None):
    """FTLM plus symmetric FTLM (Eqs. E-2-G, E-2-H) for O = dir.S: the dict of
    ``ftlm`` plus M_B_sym, M_B_sym_imag and O[r, i, j] = <v_i|O|v_j>."""
    lib = _load()
    T = default_temperatures() if T is None else np.ascontiguousarray(T, dtype=np.float64)
    nT = len(T)
    mode = {"random": 0, "basis": 1, "user": 2, "pairs": 3}[start]
    us = _cx(user_start).reshape(sys.dim, R) if mode == 2 else None
    keys = ("lnZ", "E", "C", "M_B", "M_B_imag", "M_B_sym", "M_B_sym_imag")
    out = {k: np.empty(nT) for k in keys}
    E0 = np.zeros(1)
    a = np.zeros((R, M))
    b = np.zeros((R, M))
    O = np.zeros((R, M, M), dtype=np.complex128)
    me = np.zeros(R, dtype=np.int32)
    u = None if direction is None else np.ascontiguousarray(direction, dtype=np.float64)
    cs = sys.c()
    rc = lib.oracle_sftlm(ctypes.byref(cs), R, M, seed, vec_offset, mode, basis_offset,
                          _pd(us.view(np.float64)) if us is not None else None, int(reorth), tol, _pd(u), _pd(T), nT,
                          *[_pd(out[k]) for k in keys], _pd(E0), _pd(a), _pd(b), _pd(O.view(np.float64)),
                          me.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert rc == 0, "oracle_sftlm failed"
    out.update(E0=float(E0[0]), alpha=a, beta=b, O=O, M_eff=me, T=T)
    return out


def sftlm_sums(alpha, beta, O, M_eff, g, T):
    """M_B_sym, M_B_sym_imag of Eqs. (E-2-G), (E-2-H) from per-run data."""
    lib = _load()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    R, M = a.shape
    b = np.ascontiguousarray(beta, dtype=np.float64)
    Oc = _cx(O)
    me = np.ascontiguousarray(M_eff, dtype=np.int32)
    T = np.ascontiguousarray(T, dtype=np.float64)
    mb, mbi = np.empty(len(T)), np.empty(len(T))
    assert lib.oracle_sftlm_sums(R, M, me.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _pd(a), _pd(b),
                                 _pd(Oc.view(np.float64)), float(g), _pd(T), len(T), _pd(mb), _pd(mbi)) == 0
    return mb, mbi


def num_threads() -> int:
    return int(_load().oracle_num_threads())
