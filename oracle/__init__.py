"""CPU oracle for partial modular polynomial evaluation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: ``oracle.c`` is compiled by gcc into its own shared object, and the
brute-force evaluator in ``brute.py`` uses exact Python integers.

Functions (paper Sect. 2.3: the definition of the bivariate images and the
matrix method's recurrence):
  group_keys(exps)                -> (keys[G,2], term_group[s])
  eval_direct(w)                  -> (keys, out[T,G])   O1, the definition
  eval_cells(w, t_abs, g)         -> values of chosen cells, O1 per cell
  eval_matrix(w)                  -> (keys, out[T,G])   O2, the recurrence M_i(beta^t) = m_i^t
  mulmod / addmod / powmod        -> the scalar F_p operations, for pins
  power_sums(p, z, c, t0, K)      -> a_k = sum_i c_i z_i^(t0+k), k < K
  tvandermonde_solve(p, z, a, t0) -> c with power_sums(p, z, c, t0, n) = a
                                     (Gaussian elimination; Sect. 1 interpolation)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc -O2 (no fast-math) into _build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.oracle_mulmod.restype = ctypes.c_uint64
    lib.oracle_mulmod.argtypes = [ctypes.c_uint64] * 3
    lib.oracle_addmod.restype = ctypes.c_uint64
    lib.oracle_addmod.argtypes = [ctypes.c_uint64] * 3
    lib.oracle_powmod.restype = ctypes.c_uint64
    lib.oracle_powmod.argtypes = [ctypes.c_uint64] * 3
    lib.oracle_group_keys.restype = ctypes.c_uint64
    lib.oracle_group_keys.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p, _u64p]
    ev = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, _u64p, _u32p, _u64p,
          ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p]
    lib.oracle_eval_direct.restype = ctypes.c_int
    lib.oracle_eval_direct.argtypes = ev
    lib.oracle_eval_matrix.restype = ctypes.c_int
    lib.oracle_eval_matrix.argtypes = ev
    lib.oracle_eval_cells.restype = ctypes.c_int
    lib.oracle_eval_cells.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, _u64p,
                                      _u32p, _u64p, ctypes.c_uint64, _u64p, ctypes.c_uint64,
                                      _u64p, _u64p, _u64p]
    lib.oracle_power_sums.restype = ctypes.c_int
    lib.oracle_power_sums.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, ctypes.c_uint64,
                                      ctypes.c_uint64, _u64p]
    lib.oracle_tvandermonde_solve.restype = ctypes.c_int
    lib.oracle_tvandermonde_solve.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p,
                                              ctypes.c_uint64, _u64p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def compile_variant(src_text: str, path: str):
    """Compile an altered copy of oracle.c (used by the mutation tests to show
    that the pins catch planted mistakes) and return the loaded library."""
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", path, c])
    return _configure(ctypes.CDLL(path))


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a, t):
    return a.ctypes.data_as(t)


def mulmod(a: int, b: int, p: int) -> int:
    return int(_load().oracle_mulmod(a, b, p))


def addmod(a: int, b: int, p: int) -> int:
    return int(_load().oracle_addmod(a, b, p))


def powmod(b: int, e: int, p: int) -> int:
    return int(_load().oracle_powmod(b, e, p))


def _arrays(w):
    coeffs = np.ascontiguousarray(w.coeffs, dtype=np.uint64)
    exps = np.ascontiguousarray(w.exps, dtype=np.uint32)
    beta = np.ascontiguousarray(w.beta, dtype=np.uint64)
    if beta.size == 0:
        beta = np.zeros(1, np.uint64)
    return coeffs, exps, beta


def group_keys(exps: np.ndarray):
    """(keys[G,2] uint32 in descending lex order of (d,e), term_group[s] uint64)."""
    exps = np.ascontiguousarray(exps, dtype=np.uint32)
    s, n = exps.shape
    keys = np.zeros((max(s, 1), 2), np.uint32)
    tg = np.zeros(max(s, 1), np.uint64)
    G = int(_load().oracle_group_keys(n, s, _p(exps, _u32p), _p(keys, _u32p), _p(tg, _u64p)))
    return keys[:G].copy(), tg[:s].copy()


def eval_direct(w, T=None, t0=None):
    """O1: (keys, out[T, G]) by the definition, for points t0 .. t0+T-1."""
    T = w.T if T is None else T
    t0 = w.t0 if t0 is None else t0
    coeffs, exps, beta = _arrays(w)
    keys, tg = group_keys(exps)
    G = keys.shape[0]
    out = np.zeros((T, max(G, 1)), np.uint64)
    rc = _load().oracle_eval_direct(w.p, w.n, w.s, _p(coeffs, _u64p), _p(exps, _u32p), _p(beta, _u64p),
                                    T, t0, G, _p(tg, _u64p), _p(out, _u64p))
    if rc:
        raise ValueError("oracle_eval_direct: bad arguments")
    return keys, out[:, :G].copy() if G else np.zeros((T, 0), np.uint64)


def eval_matrix(w, T=None, t0=None):
    """O2: the matrix method's recurrence, term by term (t0 >= 1)."""
    T = w.T if T is None else T
    t0 = w.t0 if t0 is None else t0
    coeffs, exps, beta = _arrays(w)
    keys, tg = group_keys(exps)
    G = keys.shape[0]
    out = np.zeros((T, max(G, 1)), np.uint64)
    rc = _load().oracle_eval_matrix(w.p, w.n, w.s, _p(coeffs, _u64p), _p(exps, _u32p), _p(beta, _u64p),
                                    T, t0, G, _p(tg, _u64p), _p(out, _u64p))
    if rc:
        raise ValueError("oracle_eval_matrix: bad arguments (t0 must be >= 1)")
    return keys, out[:, :G].copy() if G else np.zeros((T, 0), np.uint64)


class CellOracle:
    """O1 for chosen cells: value of out at absolute point t and group g."""

    def __init__(self, w):
        self.w = w
        self.coeffs, self.exps, self.beta = _arrays(w)
        self.keys, self.tg = group_keys(self.exps)
        self.G = self.keys.shape[0]

    def __call__(self, t_abs, g):
        t_abs = np.ascontiguousarray(t_abs, dtype=np.uint64)
        g = np.ascontiguousarray(g, dtype=np.uint64)
        vals = np.zeros(t_abs.shape[0], np.uint64)
        w = self.w
        rc = _load().oracle_eval_cells(w.p, w.n, w.s, _p(self.coeffs, _u64p), _p(self.exps, _u32p),
                                       _p(self.beta, _u64p), self.G, _p(self.tg, _u64p), t_abs.shape[0],
                                       _p(t_abs, _u64p), _p(g, _u64p), _p(vals, _u64p))
        if rc:
            raise ValueError("oracle_eval_cells: bad arguments")
        return vals


def eval_cells(w, t_abs, g):
    return CellOracle(w)(t_abs, g)


def power_sums(p: int, z, c, t0: int, K: int) -> np.ndarray:
    """a_k = sum_i c_i z_i^(t0+k) mod p for k = 0..K-1 (one coefficient's images)."""
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.uint64)
    a = np.zeros(max(K, 1), np.uint64)
    if _load().oracle_power_sums(p, z.shape[0], _p(z, _u64p), _p(c, _u64p), t0, K, _p(a, _u64p)):
        raise ValueError("oracle_power_sums: bad arguments")
    return a[:K].copy()


def tvandermonde_solve(p: int, z, a, t0: int):
    """c solving sum_i c_i z_i^(t0+k) = a_k, k < n = len(z); None if singular."""
    z = np.ascontiguousarray(z, dtype=np.uint64)
    a = np.ascontiguousarray(a, dtype=np.uint64)
    n = z.shape[0]
    if a.shape[0] < n:
        raise ValueError("need at least len(z) values")
    c = np.zeros(max(n, 1), np.uint64)
    rc = _load().oracle_tvandermonde_solve(p, n, _p(z, _u64p), _p(a, _u64p), t0, _p(c, _u64p))
    return None if rc else c[:n].copy()
