"""Thin Python binding of the C ABI in include/wigner.h (argument marshalling only).

Every function here checks shapes/dtypes/devices of torch tensors, allocates
outputs when they are not supplied, and passes raw device pointers and the current
CUDA stream to the library; all computation runs in the library's sm_103a kernels.
The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1002_1050_gb300.build``); if it is missing or cannot be loaded,
every call raises RuntimeError -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

WG_FP64 = 0
WG_FP32X = 1
WG_FP64S = 2
FORMS = {"fp64": WG_FP64, "fp32x": WG_FP32X, "fp64s": WG_FP64S}
WG_LMAX = 32767

_ERR = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "device allocation failed",
        -4: "bounded device wait timed out", -5: "unsupported device", -6: "not supported by this library version"}

_lock = threading.Lock()
_lib = None


class WignerError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wigner error {code} ({_ERR.get(code, '?')}): {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """Load libwigner_gb300.so (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} is missing "
                                   "(run __graft_entry__.build() or python -m paper_1002_1050_gb300.build)")
            lib = ctypes.CDLL(path)
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            sig = {
                "wigner_d_table": [I, I, I, I, P, I, P, P, P],
                "wigner_d_table_backward": [I, I, I, I, P, P, P, P],
                "wigner_conv_sum": [I, I, I, I, P, P, P, I, P, P, P],
                "wigner_conv_sum_host": [I, I, I, I, P, P, P, I, P, P],
                "wigner_conv_sum_full": [I, I, I, I, P, P, P, I, P, P, P],
                "wigner_conv_sum_multi": [I, I, I, I, I, P, P, P, I, I, I, P, P, P],
                "wigner_conv_sum_multi_tc": [I, I, I, I, I, P, P, P, P, P, P],
                "wigner_conv_sum_lmin": [I, I, I, I, P, P, P, I, D, I, P, P, P],
                "wigner_d_matrix": [I, I, I, P, P, P, P],
                "wigner_ylm": [I, I, I, P, P, P],
                "wigner_data_cube": [I, I, I, P, I, I, P, P],
                "wigner_conv_sum_backward": [I, I, I, I, P, P, P, P, P, P, P, P, I, P],
                "wigner_conv_sum_batched": [I, P, P],
                "wigner_batch_plan_create": [P, I, P, I, P],
                "wigner_batch_run": [P, I, P],
                "wigner_batch_plan_destroy": [P],
                "wigner_batch_plan_info": [P, P, P, P],
                "wigner_device_status": [P],
                "wigner_error_string": [I],
                "wigner_last_error_message": [],
                "wigner_version": [],
                "wigner_built_arch": [],
                "wigner_fma_peak": [I, I, I, I, I, P, P, P],
                "wigner_conv_sum_noalloc": [I, I, I, I, P, P, P, P, P],
                "wigner_noalloc_status": [P],
                "wigner_debug_inject_alloc_failures": [I],
                "wigner_debug_set_wait_tries": [I],
                "wigner_debug_wait_tries": [],
                "wigner_plan_create": [P, P],
                "wigner_plan_destroy": [P],
                "wigner_last_error": [],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = I
            lib.wigner_error_string.restype = ctypes.c_char_p
            lib.wigner_last_error_message.restype = ctypes.c_char_p
            lib.wigner_batch_plan_destroy.restype = None
            lib.wigner_plan_destroy.restype = None
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != 0:
        msg = load().wigner_last_error_message().decode(errors="replace")
        raise WignerError(rc, msg)


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_tensor(x, dtype, name):
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library computes on the GPU only)")
    if x.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return x


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else ctypes.c_void_p(0)


def _form(form) -> int:
    if isinstance(form, str):
        return FORMS[form]
    return int(form)


def wigner_d_table(beta: torch.Tensor, l_max: int, mb_max: int, ms_max: int, form="fp64",
                   out: torch.Tensor | None = None, counters: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """d[mb][ms][l][j] = d^l_{mb,ms}(beta_j), float64 (mb_max+1, ms_max+1, l_max+1, n_beta)."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    nb = beta.numel()
    if out is None:
        out = torch.empty((mb_max + 1, ms_max + 1, l_max + 1, nb), dtype=torch.float64, device=beta.device)
    _dev_tensor(out, torch.float64, "out")
    if tuple(out.shape) != (mb_max + 1, ms_max + 1, l_max + 1, nb):
        raise ValueError("out has the wrong shape")
    if counters is not None:
        _dev_tensor(counters, torch.int64, "counters")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_d_table(l_max, mb_max, ms_max, nb, _ptr(beta), _form(form), _ptr(out),
                                  _ptr(counters), _stream(stream)))
    return out


def wigner_d_table_backward(beta: torch.Tensor, grad_d: torch.Tensor, l_max: int, mb_max: int, ms_max: int,
                            out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """grad_beta[j] = sum grad_d[mb][ms][l][j] d/dbeta d^l_{mb,ms}(beta_j)."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    grad_d = _dev_tensor(grad_d, torch.float64, "grad_d")
    nb = beta.numel()
    if tuple(grad_d.shape) != (mb_max + 1, ms_max + 1, l_max + 1, nb):
        raise ValueError("grad_d has the wrong shape")
    if out is None:
        out = torch.empty(nb, dtype=torch.float64, device=beta.device)
    with torch.cuda.device(beta.device):
        _check(lib.wigner_d_table_backward(l_max, mb_max, ms_max, nb, _ptr(beta), _ptr(grad_d), _ptr(out),
                                           _stream(stream)))
    return out


def _conv_shapes(beta, a, b):
    if a.dim() != 2 or b.dim() != 2:
        raise ValueError("a and b must be 2-D: a[l][m_sky], b[l][m_b]")
    l_max = a.shape[0] - 1
    if b.shape[0] != l_max + 1:
        raise ValueError("a and b must have the same number of l rows")
    return l_max, b.shape[1] - 1, a.shape[1] - 1, beta.numel()


def wigner_conv_sum(beta: torch.Tensor, a: torch.Tensor, b: torch.Tensor, form="fp64",
                    out: torch.Tensor | None = None, counters: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """C[mb][ms][j] = sum_l conj(b[l][mb]) a[l][ms] d^l_{mb,ms}(beta_j), complex128."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    a = _dev_tensor(a, torch.complex128, "a")
    b = _dev_tensor(b, torch.complex128, "b")
    l_max, mb_max, ms_max, nb = _conv_shapes(beta, a, b)
    if out is None:
        out = torch.empty((mb_max + 1, ms_max + 1, nb), dtype=torch.complex128, device=beta.device)
    _dev_tensor(out, torch.complex128, "out")
    if tuple(out.shape) != (mb_max + 1, ms_max + 1, nb):
        raise ValueError("out has the wrong shape")
    if counters is not None:
        _dev_tensor(counters, torch.int64, "counters")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_conv_sum(l_max, mb_max, ms_max, nb, _ptr(beta), _ptr(a), _ptr(b), _form(form),
                                   _ptr(out), _ptr(counters), _stream(stream)))
    return out


def wigner_conv_sum_full(beta: torch.Tensor, a: torch.Tensor, b: torch.Tensor, form="fp64",
                         out: torch.Tensor | None = None, counters: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """C[mb][ms + ms_max][j] for every sky order -ms_max <= ms <= ms_max of a real sky
    (a holds m_sky >= 0), on a mirror-symmetric angle grid (beta[N-1-j] = pi - beta[j])."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    a = _dev_tensor(a, torch.complex128, "a")
    b = _dev_tensor(b, torch.complex128, "b")
    l_max, mb_max, ms_max, nb = _conv_shapes(beta, a, b)
    if out is None:
        out = torch.empty((mb_max + 1, 2 * ms_max + 1, nb), dtype=torch.complex128, device=beta.device)
    _dev_tensor(out, torch.complex128, "out")
    if tuple(out.shape) != (mb_max + 1, 2 * ms_max + 1, nb):
        raise ValueError("out has the wrong shape")
    if counters is not None:
        _dev_tensor(counters, torch.int64, "counters")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_conv_sum_full(l_max, mb_max, ms_max, nb, _ptr(beta), _ptr(a), _ptr(b), _form(form),
                                        _ptr(out), _ptr(counters), _stream(stream)))
    return out


def wigner_d_matrix(beta: torch.Tensor, l: int, m_max: int | None = None, out: torch.Tensor | None = None,
                    counters: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """d[j][m][m' + l] = d^l_{m m'}(beta_j) for 0 <= m <= m_max (default l), -l <= m' <= l."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    m_max = l if m_max is None else m_max
    shape = (beta.numel(), m_max + 1, 2 * l + 1)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=beta.device)
    _dev_tensor(out, torch.float64, "out")
    if tuple(out.shape) != shape:
        raise ValueError("out has the wrong shape")
    if counters is not None:
        _dev_tensor(counters, torch.int64, "counters")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_d_matrix(l, m_max, beta.numel(), _ptr(beta), _ptr(out), _ptr(counters),
                                   _stream(stream)))
    return out


def wigner_ylm(theta: torch.Tensor, l_max: int, m_max: int | None = None, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """y[m][l][j] = sqrt((2l+1)/(4 pi)) d^l_{m0}(theta_j): Y_l^m(theta, phi) = y[m][l][j] e^{i m phi}."""
    lib = load()
    theta = _dev_tensor(theta, torch.float64, "theta")
    m_max = l_max if m_max is None else m_max
    shape = (m_max + 1, l_max + 1, theta.numel())
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=theta.device)
    _dev_tensor(out, torch.float64, "out")
    if tuple(out.shape) != shape:
        raise ValueError("out has the wrong shape")
    with torch.cuda.device(theta.device):
        _check(lib.wigner_ylm(l_max, m_max, theta.numel(), _ptr(theta), _ptr(out), _stream(stream)))
    return out


def wigner_conv_sum_lmin(beta: torch.Tensor, a: torch.Tensor, b: torch.Tensor, offset: float, form="fp64",
                         full: bool = False, out: torch.Tensor | None = None,
                         counters: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """wigner_conv_sum (full=False) or wigner_conv_sum_full (full=True) with the l_min cut of
    Eq. lmin: each chain sums from l_min = (sqrt(m_sky^2 + m_b^2 - 2 m_sky m_b cos beta) -
    offset) / sin beta; chains cut whole are not computed (their C is 0)."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    a = _dev_tensor(a, torch.complex128, "a")
    b = _dev_tensor(b, torch.complex128, "b")
    l_max, mb_max, ms_max, nb = _conv_shapes(beta, a, b)
    shape = (mb_max + 1, 2 * ms_max + 1 if full else ms_max + 1, nb)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex128, device=beta.device)
    _dev_tensor(out, torch.complex128, "out")
    if tuple(out.shape) != shape:
        raise ValueError("out has the wrong shape")
    if counters is not None:
        _dev_tensor(counters, torch.int64, "counters")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_conv_sum_lmin(l_max, mb_max, ms_max, nb, _ptr(beta), _ptr(a), _ptr(b), _form(form),
                                        float(offset), int(bool(full)), _ptr(out), _ptr(counters),
                                        _stream(stream)))
    return out


def wigner_conv_sum_multi(beta: torch.Tensor, a: torch.Tensor, b: torch.Tensor, form="fp64",
                          sum_cols: bool = False, out: torch.Tensor | None = None,
                          counters: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """C[k][mb][ms][j] = sum_l conj(b_k[l][mb]) a[k][l][ms] d^l_{mb,ms}(beta_j) for n_col weight
    columns (Monte-Carlo skies, polarised pairs), all from one pass of the chains.

    a: (n_col, l_max+1, ms_max+1); b: (l_max+1, mb_max+1), shared by every column, or
    (n_col, l_max+1, mb_max+1), one per column.  Returns (n_col, mb_max+1, ms_max+1, n_beta),
    or with sum_cols the sum over k (the polarised total), (mb_max+1, ms_max+1, n_beta)."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    a = _dev_tensor(a, torch.complex128, "a")
    b = _dev_tensor(b, torch.complex128, "b")
    if a.dim() != 3:
        raise ValueError("a must be 3-D: a[k][l][m_sky]")
    n_col = a.shape[0]
    shared = b.dim() == 2
    if not shared and (b.dim() != 3 or b.shape[0] != n_col):
        raise ValueError("b must be b[l][m_b] (shared) or b[k][l][m_b] with a's number of columns")
    l_max, ms_max, mb_max, nb = a.shape[1] - 1, a.shape[2] - 1, b.shape[-1] - 1, beta.numel()
    if b.shape[-2] != l_max + 1:
        raise ValueError("a and b must have the same number of l rows")
    shape = (mb_max + 1, ms_max + 1, nb) if sum_cols else (n_col, mb_max + 1, ms_max + 1, nb)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex128, device=beta.device)
    _dev_tensor(out, torch.complex128, "out")
    if tuple(out.shape) != shape:
        raise ValueError("out has the wrong shape")
    if counters is not None:
        _dev_tensor(counters, torch.int64, "counters")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_conv_sum_multi(l_max, mb_max, ms_max, nb, n_col, _ptr(beta), _ptr(a), _ptr(b),
                                         int(shared), int(bool(sum_cols)), _form(form), _ptr(out), _ptr(counters),
                                         _stream(stream)))
    return out


def wigner_conv_sum_multi_tc(beta: torch.Tensor, a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None,
                             counters: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """C[k][mb][ms][j] = sum_l conj(b[l][mb]) a[k][l][ms] d^l_{mb,ms}(beta_j) for many skies a[k]
    sharing one beam b, on the tensor cores (split-bf16 slices, FP64-class accuracy).
    a: (n_col, l_max+1, ms_max+1); b: (l_max+1, mb_max+1).  Returns (n_col, mb_max+1, ms_max+1, n_beta)."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    a = _dev_tensor(a, torch.complex128, "a")
    b = _dev_tensor(b, torch.complex128, "b")
    if a.dim() != 3 or b.dim() != 2 or a.shape[1] != b.shape[0]:
        raise ValueError("a must be a[k][l][m_sky] and b b[l][m_b] with the same number of l rows")
    n_col, l_max, ms_max, mb_max, nb = a.shape[0], a.shape[1] - 1, a.shape[2] - 1, b.shape[1] - 1, beta.numel()
    shape = (n_col, mb_max + 1, ms_max + 1, nb)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex128, device=beta.device)
    _dev_tensor(out, torch.complex128, "out")
    if tuple(out.shape) != shape:
        raise ValueError("out has the wrong shape")
    if counters is not None:
        _dev_tensor(counters, torch.int64, "counters")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_conv_sum_multi_tc(l_max, mb_max, ms_max, nb, n_col, _ptr(beta), _ptr(a), _ptr(b),
                                            _ptr(out), _ptr(counters), _stream(stream)))
    return out


def fft_size(n: int) -> int:
    """Smallest integer >= n whose prime factors are 2, 3, 5 and 7 (fast FFT lengths)."""
    m = max(1, n)
    while True:
        k = m
        for p in (2, 3, 5, 7):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 1


def wigner_data_cube(c_full: torch.Tensor, n_alpha: int | None = None, n_gamma: int | None = None,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """cube[j][p][q] = sum_{m_b, m_sky} e^{-i m_b alpha_p} e^{-i m_sky gamma_q} C_{m_b m_sky}(beta_j)
    from c_full = wigner_conv_sum_full(...) (shape (mb_max+1, 2 ms_max+1, n_beta)); float64
    (n_beta, n_alpha, n_gamma), by default the smallest fast sizes without aliasing."""
    lib = load()
    c_full = _dev_tensor(c_full, torch.complex128, "c_full")
    if c_full.dim() != 3 or c_full.shape[1] % 2 != 1:
        raise ValueError("c_full must have shape (mb_max+1, 2 ms_max+1, n_beta)")
    mb_max, ms_max, nb = c_full.shape[0] - 1, (c_full.shape[1] - 1) // 2, c_full.shape[2]
    n_alpha = fft_size(2 * mb_max + 1) if n_alpha is None else n_alpha
    n_gamma = fft_size(2 * ms_max + 1) if n_gamma is None else n_gamma
    if out is None:
        out = torch.empty((nb, n_alpha, n_gamma), dtype=torch.float64, device=c_full.device)
    _dev_tensor(out, torch.float64, "out")
    if tuple(out.shape) != (nb, n_alpha, n_gamma):
        raise ValueError("out has the wrong shape")
    with torch.cuda.device(c_full.device):
        _check(lib.wigner_data_cube(mb_max, ms_max, nb, _ptr(c_full), n_alpha, n_gamma, _ptr(out),
                                    _stream(stream)))
    return out


def _host_tensor(x, dtype, name):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(x)
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a numpy array or a CPU torch.Tensor")
    if x.is_cuda:
        raise ValueError(f"{name} must be in host memory (use wigner_conv_sum for device tensors)")
    if x.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return x


def wigner_conv_sum_host(beta, a, b, form="fp64", out=None, stream=None, sync=True):
    """wigner_conv_sum on host buffers (numpy arrays or CPU tensors; pinned memory lets the
    copies overlap the computation).  Returns out, a CPU complex128 tensor
    (mb_max+1, ms_max+1, n_beta); with sync=False the caller synchronises the stream
    before reading it."""
    lib = load()
    beta = _host_tensor(beta, torch.float64, "beta")
    a = _host_tensor(a, torch.complex128, "a")
    b = _host_tensor(b, torch.complex128, "b")
    if a.dim() != 2 or b.dim() != 2 or beta.dim() != 1 or a.shape[0] != b.shape[0]:
        raise ValueError("expected beta (n_beta,), a (l_max+1, ms_max+1), b (l_max+1, mb_max+1)")
    l_max, ms_max, mb_max, nb = a.shape[0] - 1, a.shape[1] - 1, b.shape[1] - 1, beta.numel()
    if out is None:
        out = torch.empty((mb_max + 1, ms_max + 1, nb), dtype=torch.complex128, pin_memory=torch.cuda.is_available())
    out = _host_tensor(out, torch.complex128, "out")
    if tuple(out.shape) != (mb_max + 1, ms_max + 1, nb):
        raise ValueError("out has the wrong shape")
    s = _stream(stream)
    _check(lib.wigner_conv_sum_host(l_max, mb_max, ms_max, nb, _ptr(beta), _ptr(a), _ptr(b), _form(form),
                                    _ptr(out), s))
    if sync:
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
    return out


def wigner_conv_sum_backward(beta, a, b, c_fwd, grad_c, need_a=True, need_b=True, need_beta=True,
                             stream=None):
    """(grad_a, grad_b, grad_beta) for a real loss with dL/dC = grad_c (PyTorch convention)."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    a = _dev_tensor(a, torch.complex128, "a")
    b = _dev_tensor(b, torch.complex128, "b")
    grad_c = _dev_tensor(grad_c, torch.complex128, "grad_c")
    l_max, mb_max, ms_max, nb = _conv_shapes(beta, a, b)
    if c_fwd is not None:
        _dev_tensor(c_fwd, torch.complex128, "c_fwd")
    ga = torch.empty_like(a) if need_a else None
    gb = torch.empty_like(b) if need_b else None
    gbeta = torch.empty_like(beta) if need_beta else None
    with torch.cuda.device(beta.device):
        _check(lib.wigner_conv_sum_backward(l_max, mb_max, ms_max, nb, _ptr(beta), _ptr(a), _ptr(b), _ptr(c_fwd),
                                            _ptr(grad_c), _ptr(ga), _ptr(gb), _ptr(gbeta), WG_FP64,
                                            _stream(stream)))
    return ga, gb, gbeta


def wigner_conv_sum_noalloc(beta: torch.Tensor, a: torch.Tensor, b: torch.Tensor, out: torch.Tensor,
                            stream=None) -> torch.Tensor:
    """wigner_conv_sum (FP64) through the allocation-free entry point; `out` must be supplied
    (complex128, (mb_max+1, ms_max+1, n_beta)) and l_max <= 8192."""
    lib = load()
    beta = _dev_tensor(beta, torch.float64, "beta")
    a = _dev_tensor(a, torch.complex128, "a")
    b = _dev_tensor(b, torch.complex128, "b")
    out = _dev_tensor(out, torch.complex128, "out")
    l_max, mb_max, ms_max, nb = _conv_shapes(beta, a, b)
    if tuple(out.shape) != (mb_max + 1, ms_max + 1, nb):
        raise ValueError("out has the wrong shape")
    with torch.cuda.device(beta.device):
        _check(lib.wigner_conv_sum_noalloc(l_max, mb_max, ms_max, nb, _ptr(beta), _ptr(a), _ptr(b), _ptr(out),
                                           _stream(stream)))
    return out


class WgInstance(ctypes.Structure):
    """Mirror of the C ABI's wg_instance."""
    _fields_ = [("l_max", ctypes.c_int), ("mb_max", ctypes.c_int), ("ms_max", ctypes.c_int),
                ("n_beta", ctypes.c_int), ("form", ctypes.c_int), ("beta", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("c_out", ctypes.c_void_p)]


def _instances(problems):
    """problems: list of (beta, a, b, form, out) with CUDA tensors (out may be None)."""
    arr = (WgInstance * len(problems))()
    outs, keep = [], []
    for i, (beta, a, b, form, out) in enumerate(problems):
        beta = _dev_tensor(beta, torch.float64, "beta")
        a = _dev_tensor(a, torch.complex128, "a")
        b = _dev_tensor(b, torch.complex128, "b")
        l_max, mb_max, ms_max, nb = _conv_shapes(beta, a, b)
        if out is None:
            out = torch.empty((mb_max + 1, ms_max + 1, nb), dtype=torch.complex128, device=beta.device)
        _dev_tensor(out, torch.complex128, "out")
        if tuple(out.shape) != (mb_max + 1, ms_max + 1, nb):
            raise ValueError(f"instance {i}: out has the wrong shape")
        arr[i] = WgInstance(l_max, mb_max, ms_max, nb, _form(form), beta.data_ptr(), a.data_ptr(), b.data_ptr(),
                            out.data_ptr())
        outs.append(out)
        keep.extend([beta, a, b, out])
    return arr, outs, keep


class BatchPlan:
    """A batch of uneven fused sums run by one persistent launch (wigner_batch_plan_*).

    The tensors passed in are kept alive by the plan (the device code holds their pointers).
    """

    def __init__(self, problems, autotune: bool = False, stream=None):
        lib = load()
        self._arr, self.outputs, self._keep = _instances(problems)
        self._plan = ctypes.c_void_p(0)
        _check(lib.wigner_batch_plan_create(ctypes.byref(self._plan), len(problems), self._arr, int(autotune),
                                            _stream(stream)))

    def run(self, use_graph: bool = False, stream=None):
        _check(load().wigner_batch_run(self._plan, int(use_graph), _stream(stream)))
        return self.outputs

    def info(self):
        v, n, g = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(load().wigner_batch_plan_info(self._plan, ctypes.byref(v), ctypes.byref(n), ctypes.byref(g)))
        return {"variant": v.value, "n_items": n.value, "grid": g.value}

    def close(self):
        if self._plan:
            load().wigner_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wigner_conv_sum_batched(problems, stream=None):
    """Run (beta, a, b, form, out) problems in one persistent launch; returns the outputs.
    Blocks until the batch has finished."""
    arr, outs, _keep = _instances(problems)
    _check(load().wigner_conv_sum_batched(len(problems), arr, _stream(stream)))
    return outs


class WgParams(ctypes.Structure):
    _fields_ = [("l_max_cap", ctypes.c_int), ("mb_max_cap", ctypes.c_int), ("ms_max_cap", ctypes.c_int),
                ("n_beta_cap", ctypes.c_int), ("reserve_backward", ctypes.c_int)]


class Plan:
    """Reserve tables (and optionally the adjoints' workspace) so that calls within the
    caps allocate nothing -- e.g. to capture them in a CUDA graph (wigner_plan_create)."""

    def __init__(self, l_max_cap: int, mb_max_cap: int = 0, ms_max_cap: int = 0, n_beta_cap: int = 0,
                 reserve_backward: bool = False):
        lib = load()
        self._h = ctypes.c_void_p(0)
        prm = WgParams(l_max_cap, mb_max_cap, ms_max_cap, n_beta_cap, int(reserve_backward))
        _check(lib.wigner_plan_create(ctypes.byref(self._h), ctypes.byref(prm)))

    def close(self):
        if self._h:
            load().wigner_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wigner_device_status(stream=None) -> int:
    """Synchronise the stream; return (and clear) the library's device status code."""
    return int(load().wigner_device_status(_stream(stream)))


def check_device_status(stream=None):
    rc = wigner_device_status(stream)
    _check(rc)


def wigner_fma_peak(pipe: int, blocks: int, threads: int, iters: int, chains: int = 8, stream=None):
    """Launch the FMA microbenchmark (`chains` independent FMA chains per thread); returns
    (sink tensor, FMA lane-operations)."""
    lib = load()
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    ops = ctypes.c_ulonglong(0)
    _check(lib.wigner_fma_peak(pipe, chains, blocks, threads, iters, _ptr(sink), ctypes.byref(ops),
                               _stream(stream)))
    return sink, int(ops.value)


def wigner_noalloc_status(stream=None) -> int:
    """Synchronise the stream; return (and clear) the status code of wigner_conv_sum_noalloc
    on the current device (allocates nothing)."""
    return int(load().wigner_noalloc_status(_stream(stream)))


def debug_inject_alloc_failures(n: int):
    """Test hook: the library's next n device allocations fail as if out of memory."""
    _check(load().wigner_debug_inject_alloc_failures(int(n)))


def debug_set_wait_tries(tries: int) -> int:
    """Test hook: tries of each TMA wait of the fused sums launched from now on (0 gives
    up at once; the default is 2**20).  Returns the previous value."""
    lib = load()
    old = int(lib.wigner_debug_wait_tries())
    _check(lib.wigner_debug_set_wait_tries(int(tries)))
    return old


def exported_symbols():
    """Names the binding expects the library to export (for the ABI test)."""
    return ["wigner_d_table", "wigner_d_table_backward", "wigner_conv_sum", "wigner_conv_sum_backward",
            "wigner_conv_sum_batched", "wigner_batch_plan_create", "wigner_batch_run",
            "wigner_batch_plan_destroy", "wigner_device_status", "wigner_error_string",
            "wigner_last_error_message", "wigner_version", "wigner_built_arch", "wigner_fma_peak",
            "wigner_conv_sum_noalloc", "wigner_batch_plan_info", "wigner_plan_create", "wigner_plan_destroy",
            "wigner_last_error", "wigner_conv_sum_host", "wigner_conv_sum_full", "wigner_data_cube",
            "wigner_conv_sum_multi", "wigner_conv_sum_lmin", "wigner_d_matrix", "wigner_ylm",
            "wigner_noalloc_status", "wigner_debug_inject_alloc_failures", "wigner_debug_set_wait_tries",
            "wigner_debug_wait_tries", "wigner_conv_sum_multi_tc"]
