"""The allocation-free entry point wigner_conv_sum_noalloc, called through the C ABI.

It is meant for callers that must not let the library allocate device memory (stream
capture in progress, an application-owned memory pool, real-time loops).  It runs the
same fused FP64 kernel as wigner_conv_sum with its constant tables in a fixed array
inside the library; the test checks two consecutive calls against wigner_conv_sum
within the FP64 tolerance of the other parity tests (1e-11), and that the second call
leaves the device's free memory unchanged.  This file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import wigner as W
    return W, W.load()


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _call_noalloc(raw, L, MB, MS, beta, a, b, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return raw.wigner_conv_sum_noalloc(L, MB, MS, beta.numel(), ctypes.c_void_p(beta.data_ptr()),
                                       ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_allocating_entry_point_twice(lib):
    W, raw = lib
    L, MB, MS, NB = 300, 8, 300, 600
    beta = _cuda(I.beta_gauss_legendre(NB)[0])
    a = _cuda(I.sky_alm(L, MS, 3))
    b = _cuda(I.beam_blm(L, MB, fwhm=0.03))
    ref = W.wigner_conv_sum(beta, a, b)
    W.check_device_status()
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full((MB + 1, MS + 1, NB), complex(math.nan, math.nan), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call_noalloc(raw, L, MB, MS, beta, a, b, out)
        assert rc == 0, raw.wigner_last_error_message()
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:  # after the per-device set-up of the first call
            assert free_after == free_before
        err = float((out - ref).abs().max())
        assert err <= TOL, (call, err)


def test_noalloc_rejects_too_large_l_max(lib):
    _, raw = lib
    beta = torch.zeros(4, dtype=torch.float64, device="cuda")
    big = 8193  # one more than the fixed tables hold
    a = torch.zeros((big + 1, 2), dtype=torch.complex128, device="cuda")
    b = torch.zeros((big + 1, 2), dtype=torch.complex128, device="cuda")
    out = torch.zeros((2, 2, 4), dtype=torch.complex128, device="cuda")
    rc = _call_noalloc(raw, big, 1, 1, beta, a, b, out)
    assert rc == -1
    assert b"8192" in raw.wigner_last_error_message()
