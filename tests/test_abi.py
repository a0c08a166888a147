"""CPU checks of the C-ABI library: it builds, loads, exports every declared symbol,
and rejects invalid arguments on the host (no GPU needed for any of this)."""
import ctypes
import os
import re

import pytest

from paper_1002_1050_gb300 import build as B
from paper_1002_1050_gb300 import wigner as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "wigner.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(wigner_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return W.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("wigner_d_table", "wigner_d_table_backward", "wigner_conv_sum", "wigner_conv_sum_backward",
                 "wigner_conv_sum_batched", "wigner_device_status", "wigner_fma_peak"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(W.exported_symbols()) == set(_declared_functions())


def test_version_and_arch(lib):
    assert lib.wigner_version() >= 1
    assert lib.wigner_built_arch() == 1003
    assert lib.wigner_error_string(0) == b"ok"
    assert lib.wigner_error_string(-1) == b"invalid argument"


P = ctypes.c_void_p
FAKE = P(0x1000)  # never dereferenced: validation fails before any device access


@pytest.mark.parametrize("l_max,mb,ms,nb", [(-1, 0, 0, 1), (4, 5, 0, 1), (4, 0, 5, 1), (4, -1, 0, 1),
                                           (4, 0, 0, -3), (W.WG_LMAX + 1, 0, 0, 1)])
def test_bad_orders_rejected(lib, l_max, mb, ms, nb):
    assert lib.wigner_d_table(l_max, mb, ms, nb, FAKE, 0, FAKE, None, None) == -1
    assert lib.wigner_conv_sum(l_max, mb, ms, nb, FAKE, FAKE, FAKE, 0, FAKE, None, None) == -1


def test_null_and_misaligned_pointers_rejected(lib):
    assert lib.wigner_conv_sum(8, 2, 8, 4, None, FAKE, FAKE, 0, FAKE, None, None) == -1
    assert b"beta" in lib.wigner_last_error_message()
    assert lib.wigner_conv_sum(8, 2, 8, 4, FAKE, P(0x1008), FAKE, 0, FAKE, None, None) == -1
    assert b"aligned" in lib.wigner_last_error_message()
    assert lib.wigner_d_table(8, 2, 8, 4, FAKE, 0, None, None, None) == -1
    assert lib.wigner_d_table(8, 2, 8, 4, FAKE, 7, FAKE, None, None) == -1  # unknown form
    assert lib.wigner_fma_peak(3, 8, 1, 32, 1, FAKE, None, None) == -1  # unknown pipe
    assert lib.wigner_fma_peak(0, 3, 1, 32, 1, FAKE, None, None) == -1  # chains not a power of two <= 16


def test_empty_angle_set_is_a_noop(lib):
    # n_beta = 0: nothing to compute, no device touched
    assert lib.wigner_d_table(8, 2, 8, 0, None, 0, None, None, None) == 0
    assert lib.wigner_conv_sum(8, 2, 8, 0, None, FAKE, FAKE, 0, None, None, None) == 0


def test_binding_rejects_cpu_tensors():
    import torch
    with pytest.raises(ValueError):
        W.wigner_d_table(torch.zeros(3, dtype=torch.float64), 4, 1, 4)


def test_plan_and_last_error_validation(lib):
    assert lib.wigner_plan_create(None, None) == -1
    assert lib.wigner_last_error() == -1
    h = ctypes.c_void_p(0)
    prm = W.WgParams(-1, 0, 0, 0, 0)
    assert lib.wigner_plan_create(ctypes.byref(h), ctypes.byref(prm)) == -1
    assert not h.value
    lib.wigner_plan_destroy(None)  # NULL is accepted


def test_host_entry_point_validation(lib):
    H = ctypes.c_void_p(0x1000)  # never touched: validation fails first
    assert lib.wigner_conv_sum_host(8, 2, 8, 4, None, H, H, 0, H, None) == -1
    assert lib.wigner_conv_sum_host(8, 9, 8, 4, H, H, H, 0, H, None) == -1   # mb_max > l_max
    assert lib.wigner_conv_sum_host(8, 2, 8, 4, H, H, H, 5, H, None) == -1   # unknown form
    assert lib.wigner_conv_sum_host(8, 2, 8, 0, None, None, None, 0, None, None) == 0  # nothing to do


def test_multi_entry_point_validation(lib):
    # (l_max, mb, ms, nb, n_col, beta, a, b, b_shared, sum_cols, form, c, counters, stream)
    assert lib.wigner_conv_sum_multi(8, 9, 8, 4, 2, FAKE, FAKE, FAKE, 1, 0, 0, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_multi(8, 2, 8, 4, -1, FAKE, FAKE, FAKE, 1, 0, 0, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_multi(8, 2, 8, 4, 2, None, FAKE, FAKE, 1, 0, 0, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_multi(8, 2, 8, 4, 2, FAKE, P(0x1008), FAKE, 1, 0, 0, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_multi(8, 2, 8, 4, 2, FAKE, FAKE, FAKE, 1, 0, 1, FAKE, None, None) == -6  # FP32X
    assert lib.wigner_conv_sum_multi(8, 2, 8, 4, 2, FAKE, FAKE, FAKE, 1, 0, 5, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_multi(8, 2, 8, 0, 2, None, None, None, 1, 0, 0, None, None, None) == 0
    assert lib.wigner_conv_sum_multi(8, 2, 8, 4, 0, FAKE, None, None, 1, 0, 0, FAKE, None, None) == 0


def test_lmin_entry_point_validation(lib):
    D = ctypes.c_double
    # (l_max, mb, ms, nb, beta, a, b, form, offset, full, c, counters, stream)
    assert lib.wigner_conv_sum_lmin(8, 9, 8, 4, FAKE, FAKE, FAKE, 0, D(10.0), 0, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_lmin(8, 2, 8, 4, FAKE, FAKE, FAKE, 0, D(float("nan")), 0, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_lmin(8, 2, 8, 4, FAKE, FAKE, FAKE, 1, D(10.0), 0, FAKE, None, None) == -6
    assert lib.wigner_conv_sum_lmin(8, 2, 8, 4, None, FAKE, FAKE, 0, D(10.0), 1, FAKE, None, None) == -1
    assert lib.wigner_conv_sum_lmin(8, 2, 8, 0, None, None, None, 0, D(10.0), 1, None, None, None) == 0


def test_matrix_and_ylm_validation(lib):
    assert lib.wigner_d_matrix(-1, 0, 4, FAKE, FAKE, None, None) == -1
    assert lib.wigner_d_matrix(5, 6, 4, FAKE, FAKE, None, None) == -1      # m_max > l
    assert lib.wigner_d_matrix(5, 2, 4, None, FAKE, None, None) == -1
    assert lib.wigner_d_matrix(5, 2, 4, FAKE, P(0x1004), None, None) == -1  # misaligned
    assert lib.wigner_d_matrix(5, 2, 0, None, None, None, None) == 0
    assert lib.wigner_ylm(5, 6, 4, FAKE, FAKE, None) == -1
    assert lib.wigner_ylm(5, 2, 4, None, FAKE, None) == -1
    assert lib.wigner_ylm(5, 2, 0, None, None, None) == 0


def test_debug_hooks_validate_and_round_trip(lib):
    # host-side knobs only: no device is touched
    assert lib.wigner_debug_inject_alloc_failures(-1) == -1
    assert lib.wigner_debug_set_wait_tries(-5) == -1
    old = lib.wigner_debug_wait_tries()
    assert old == 1 << 20
    assert lib.wigner_debug_set_wait_tries(7) == 0 and lib.wigner_debug_wait_tries() == 7
    assert lib.wigner_debug_set_wait_tries(old) == 0 and lib.wigner_debug_wait_tries() == old
    assert lib.wigner_debug_inject_alloc_failures(0) == 0
