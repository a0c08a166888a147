"""ctypes wrapper around the plain C oracle (wigner_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product path never imports this module.

All arrays are numpy float64 / complex128 in the layouts documented in
wigner_oracle.c.  `build()` compiles the library in place with gcc (OpenMP,
-O2 -ffp-contract=off, no fast-math).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wigner_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_wigner.so")
_lock = threading.Lock()
_lib = None


def _lib_path(plant: int) -> str:
    return _LIB_PATH if plant == 0 else os.path.join(_OUT_DIR, f"liboracle_wigner_plant{plant}.so")


def build(force: bool = False, plant: int = 0) -> str:
    """Compile the oracle shared library (idempotent unless the source is newer).

    plant > 0 builds a separate copy with one deliberate mistake (ORACLE_PLANT),
    used only by the test that checks the pins catch such mistakes.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    path = _lib_path(plant)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-std=c11", "-Wall", f"-DORACLE_PLANT={int(plant)}", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _open(path):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.oracle_d_table.argtypes = [I, I, I, I, P, I, P]
    lib.oracle_d_table.restype = I
    lib.oracle_d_column.argtypes = [I, I, I, I, P, P]
    lib.oracle_d_column.restype = I
    lib.oracle_d_single.argtypes = [I, I, I, ctypes.c_double]
    lib.oracle_d_single.restype = ctypes.c_double
    lib.oracle_conv_sum.argtypes = [I, I, I, I, P, P, P, P]
    lib.oracle_conv_sum.restype = I
    lib.oracle_conv_sum_full.argtypes = [I, I, I, I, P, P, P, P]
    lib.oracle_conv_sum_full.restype = I
    lib.oracle_conv_sum_full_sampled.argtypes = [I, I, I, I, P, P, P, I, P, P]
    lib.oracle_conv_sum_full_sampled.restype = I
    lib.oracle_conv_sum_sampled.argtypes = [I, I, I, I, P, P, P, I, P, P]
    lib.oracle_conv_sum_sampled.restype = I
    D = ctypes.c_double
    lib.oracle_conv_sum_lmin.argtypes = [I, I, I, I, P, P, P, D, P]
    lib.oracle_conv_sum_lmin.restype = I
    lib.oracle_conv_sum_full_lmin.argtypes = [I, I, I, I, P, P, P, D, P]
    lib.oracle_conv_sum_full_lmin.restype = I
    lib.oracle_conv_sum_full_sampled_lmin.argtypes = [I, I, I, I, P, P, P, I, P, D, P]
    lib.oracle_conv_sum_full_sampled_lmin.restype = I
    lib.oracle_d_matrix.argtypes = [I, I, I, P, P]
    lib.oracle_d_matrix.restype = I
    lib.oracle_l_first.argtypes = [I, I, I, D, D]
    lib.oracle_l_first.restype = I
    lib.oracle_conv_grad.argtypes = [I, I, I, I, P, P, P, P, P, P, P]
    lib.oracle_conv_grad.restype = I
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = I
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _open(build())
    return _lib


class Planted:
    """A copy of the oracle compiled with ORACLE_PLANT=k (test of the pins only)."""

    def __init__(self, plant: int):
        self._lib = _open(build(plant=plant))

    def d_table(self, *args, **kw):
        return d_table(*args, _lib=self._lib, **kw)

    def conv_sum(self, *args, **kw):
        return conv_sum(*args, _lib=self._lib, **kw)

    def d_single(self, *args, **kw):
        return d_single(*args, _lib=self._lib, **kw)

    def conv_sum_full(self, *args, **kw):
        return conv_sum_full(*args, _lib=self._lib, **kw)

    def l_first(self, *args, **kw):
        return l_first(*args, _lib=self._lib, **kw)

    def d_matrix(self, *args, **kw):
        return d_matrix(*args, _lib=self._lib, **kw)


def _ptr(x):
    return None if x is None else x.ctypes.data_as(ctypes.c_void_p)


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _c128(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def d_table(l_max: int, mb_max: int, ms_max: int, beta, scaling: bool = True, _lib=None) -> np.ndarray:
    """d[mb][ms][l][j] = d^l_{mb,ms}(beta_j); zero where l < max(mb, ms)."""
    lib = _lib or _load()
    beta = _f64(beta)
    out = np.empty((mb_max + 1, ms_max + 1, l_max + 1, beta.size), dtype=np.float64)
    rc = lib.oracle_d_table(l_max, mb_max, ms_max, beta.size, _ptr(beta), int(scaling), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_d_table: invalid arguments")
    return out


def d_column(l_max: int, mb: int, ms: int, beta) -> np.ndarray:
    """d[l][j] = d^l_{mb,ms}(beta_j) for one chain column, l = 0..l_max."""
    lib = _load()
    beta = _f64(beta)
    out = np.empty((l_max + 1, beta.size), dtype=np.float64)
    if lib.oracle_d_column(l_max, mb, ms, beta.size, _ptr(beta), _ptr(out)) != 0:
        raise ValueError("oracle_d_column: invalid arguments")
    return out


def d_matrix(l: int, m_max: int, beta, _lib=None) -> np.ndarray:
    """d[m][m' + l][j] = d^l_{m m'}(beta_j) for 0 <= m <= m_max, -l <= m' <= l: each element
    the end of its own l-chain (the definition through the pinned chain code)."""
    lib = _lib or _load()
    beta = _f64(beta)
    out = np.empty((m_max + 1, 2 * l + 1, beta.size), dtype=np.float64)
    if lib.oracle_d_matrix(l, m_max, beta.size, _ptr(beta), _ptr(out)) != 0:
        raise ValueError("oracle_d_matrix: invalid arguments")
    return out


def d_single(l: int, m: int, mp: int, beta: float, _lib=None) -> float:
    """One element d^l_{m m'}(beta), 0 <= m, m' <= l."""
    return float((_lib or _load()).oracle_d_single(l, m, mp, float(beta)))


def conv_sum(l_max: int, mb_max: int, ms_max: int, beta, a, b, _lib=None, offset=None) -> np.ndarray:
    """C[mb][ms][j] = sum_l conj(b[l][mb]) a[l][ms] d^l_{mb ms}(beta_j), complex128.
    offset: the sum starts at the l_min of Eq. lmin for that offset (None: no cut)."""
    lib = _lib or _load()
    beta, a, b = _f64(beta), _c128(a), _c128(b)
    assert a.shape == (l_max + 1, ms_max + 1) and b.shape == (l_max + 1, mb_max + 1)
    out = np.empty((mb_max + 1, ms_max + 1, beta.size), dtype=np.complex128)
    if offset is not None:
        rc = lib.oracle_conv_sum_lmin(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a), _ptr(b),
                                      float(offset), _ptr(out))
    else:
        rc = lib.oracle_conv_sum(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a), _ptr(b), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_conv_sum: invalid arguments")
    return out


def conv_sum_full(l_max: int, mb_max: int, ms_max: int, beta, a, b, _lib=None, offset=None) -> np.ndarray:
    """C[mb][ms + ms_max][j] for every sky order -ms_max <= ms <= ms_max of a real sky
    (s_{l,-m} = (-1)^m conj(a[l][m])); each negative order runs its own chain.
    offset: with the l_min cut of Eq. lmin (None: no cut)."""
    lib = _lib or _load()
    beta, a, b = _f64(beta), _c128(a), _c128(b)
    assert a.shape == (l_max + 1, ms_max + 1) and b.shape == (l_max + 1, mb_max + 1)
    out = np.empty((mb_max + 1, 2 * ms_max + 1, beta.size), dtype=np.complex128)
    if offset is not None:
        rc = lib.oracle_conv_sum_full_lmin(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a), _ptr(b),
                                           float(offset), _ptr(out))
    else:
        rc = lib.oracle_conv_sum_full(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a), _ptr(b),
                                      _ptr(out))
    if rc != 0:
        raise ValueError("oracle_conv_sum_full: invalid arguments")
    return out


def conv_sum_full_sampled(l_max: int, mb_max: int, ms_max: int, beta, a, b, idx, offset=None) -> np.ndarray:
    """conv_sum_full at the (mb, ms, j) triples of idx (ms may be negative), complex128 [n]."""
    lib = _load()
    beta, a, b = _f64(beta), _c128(a), _c128(b)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(-1, 3))
    out = np.empty(idx.shape[0], dtype=np.complex128)
    if offset is not None:
        rc = lib.oracle_conv_sum_full_sampled_lmin(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a),
                                                   _ptr(b), idx.shape[0], _ptr(idx), float(offset), _ptr(out))
    else:
        rc = lib.oracle_conv_sum_full_sampled(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a), _ptr(b),
                                              idx.shape[0], _ptr(idx), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_conv_sum_full_sampled: invalid arguments")
    return out


def conv_sum_sampled(l_max: int, mb_max: int, ms_max: int, beta, a, b, idx) -> np.ndarray:
    """C at the (mb, ms, j) triples of idx (shape [n, 3]), complex128 [n]."""
    lib = _load()
    beta, a, b = _f64(beta), _c128(a), _c128(b)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(-1, 3))
    out = np.empty(idx.shape[0], dtype=np.complex128)
    rc = lib.oracle_conv_sum_sampled(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a), _ptr(b),
                                     idx.shape[0], _ptr(idx), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_conv_sum_sampled: invalid arguments")
    return out


def l_first(l_max: int, mb: int, mp: int, beta: float, offset: float, _lib=None) -> int:
    """First l of the sum of chain (mb, mp, beta) under the l_min cut of Eq. lmin
    (max(|mb|, |mp|) if nothing is cut, l_max + 1 if the whole chain is)."""
    return int((_lib or _load()).oracle_l_first(l_max, mb, mp, float(beta), float(offset)))


def conv_sum_multi(l_max: int, mb_max: int, ms_max: int, beta, a, b, sum_cols: bool = False) -> np.ndarray:
    """Eq. convdef for several weight columns (the polarised pairs of the footnote of Sec. 4.1,
    or Monte-Carlo skies): column k is conv_sum with a[k] and b (one beam) or b[k].
    Returns (n_col, mb+1, ms+1, n_beta), or with sum_cols the sum over the columns."""
    a = np.asarray(a)
    b = np.asarray(b)
    cols = [conv_sum(l_max, mb_max, ms_max, beta, a[k], b if b.ndim == 2 else b[k]) for k in range(a.shape[0])]
    if sum_cols:
        out = np.zeros((mb_max + 1, ms_max + 1, np.size(beta)), dtype=np.complex128)
        for c in cols:
            out += c
        return out
    return np.array(cols).reshape(a.shape[0], mb_max + 1, ms_max + 1, np.size(beta))


def conv_grad(l_max: int, mb_max: int, ms_max: int, beta, a, b, grad_c,
              want_a: bool = True, want_b: bool = True, want_beta: bool = True):
    """(grad_a, grad_b, grad_beta) of a real loss whose gradient w.r.t. C is grad_c."""
    lib = _load()
    beta, a, b, g = _f64(beta), _c128(a), _c128(b), _c128(grad_c)
    assert g.shape == (mb_max + 1, ms_max + 1, beta.size)
    ga = np.empty_like(a) if want_a else None
    gb = np.empty_like(b) if want_b else None
    gbeta = np.empty_like(beta) if want_beta else None
    rc = lib.oracle_conv_grad(l_max, mb_max, ms_max, beta.size, _ptr(beta), _ptr(a), _ptr(b), _ptr(g),
                              _ptr(ga), _ptr(gb), _ptr(gbeta))
    if rc != 0:
        raise ValueError("oracle_conv_grad: invalid arguments")
    return ga, gb, gbeta


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS or all host cores)."""
    return int(_load().oracle_num_threads())
