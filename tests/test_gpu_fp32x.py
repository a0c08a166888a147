"""GPU parity of the FP32 form (float recursion with an int32 exponent carry).

Bars: d-table within 2e-4 absolute of the FP64 oracle; C within 1e-4 relative L2 of
the FP64 kernel and of the FP64 oracle.  The full 8192/16/8192/8192-angle sum is run
in full; its FP64 comparison uses every 16th angle (the FP64 kernel needs ~40 s for
all of them) and the oracle checks sampled outputs.
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import wigner
    wigner.load()
    return wigner


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel_l2(x, ref):
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


def test_dtable_fp32x_l256(W):
    L, MB, MS, beta, _, _ = I.make_config("dtable_l256")
    d = W.wigner_d_table(_cuda(beta), L, MB, MS, form="fp32x").cpu().numpy()
    W.check_device_status()
    ref = O.d_table(L, MB, MS, beta)
    err = float(np.max(np.abs(d - ref)))
    assert err <= 2e-4, err


@pytest.mark.parametrize("NB", [7, 300])
def test_dtable_fp32x_poles_and_turning_points(W, NB):
    """Angles near both poles and across pi/2; orders whose turning point is inside the range."""
    L, MB, MS = 1500, 16, 1500
    beta = np.concatenate([[0.0, 1e-4, 3e-4, math.pi / 2, math.pi - 3e-4, math.pi],
                           I.beta_uniform(max(NB - 6, 1), 1e-3, math.pi - 1e-3, 2)])[:NB]
    cols = [(0, 0), (16, 16), (3, 700), (16, 1499), (0, 1500)]
    d = W.wigner_d_table(_cuda(beta), L, MB, MS, form="fp32x")
    W.check_device_status()
    for mb, ms in cols:
        ref = O.d_column(L, mb, ms, beta)
        got = d[mb, ms].cpu().numpy()
        assert float(np.max(np.abs(got - ref))) <= 2e-4, (mb, ms)


@pytest.mark.parametrize("L,MB,MS,NB", [(64, 4, 64, 300), (200, 8, 120, 513), (700, 16, 700, 97)])
def test_conv_fp32x_small(W, L, MB, MS, NB):
    beta = I.beta_gauss_legendre(NB)[0]
    a = I.sky_alm(L, MS, 5)
    rng = np.random.default_rng(6)
    b = I.beam_blm(L, MB, fwhm=0.05) + 0.05j * rng.standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form="fp32x").cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum(L, MB, MS, beta, a, b)
    assert _rel_l2(C, ref) <= 1e-4
    assert np.all(np.isfinite(C))


def test_conv_fp32x_weights_outside_float_range(W):
    """Columns whose weights lie far outside float's range (a sky column scaled by 1e-80,
    beam orders by 1e-70 and 1e+60): each non-zero column of C keeps its relative accuracy, as the
    weights enter the float recursion with a per-column power-of-two scale."""
    L, MB, MS, NB = 300, 4, 300, 257
    beta = I.beta_gauss_legendre(NB)[0]
    a = I.sky_alm(L, MS, 21)
    b = I.beam_blm(L, MB, fwhm=0.03)
    a[:, 7] *= 1e-80
    b[:, 2] *= 1e-70
    b[:, 4] *= 1e60
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form="fp32x").cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum(L, MB, MS, beta, a, b)
    assert np.all(np.isfinite(C))
    for mb in range(MB + 1):
        for ms in (0, 7, 150, 300):
            if not np.any(ref[mb, ms]):  # the beam's odd orders are zero
                assert not np.any(C[mb, ms]), (mb, ms)
            else:
                assert _rel_l2(C[mb, ms], ref[mb, ms]) <= 1e-4, (mb, ms)


def test_conv_fp32x_unsorted_angles_with_poles(W):
    """Angles in random order, both poles and pi/2 included: threads hold chains on both
    sides of pi/2 (each chain picks its own K coefficient) and scaled and plain chains
    share warps; also two angle chunks of 512."""
    L, MB, MS, NB = 900, 6, 900, 700
    beta = np.concatenate([[0.0, 1e-4, math.pi / 2, math.pi - 1e-4, math.pi],
                           I.beta_uniform(NB - 5, 1e-3, math.pi - 1e-3, 9)])
    np.random.default_rng(10).shuffle(beta)
    a = I.sky_alm(L, MS, 11)
    b = I.beam_blm(L, MB, fwhm=0.02)
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form="fp32x").cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum(L, MB, MS, beta, a, b)
    assert _rel_l2(C, ref) <= 1e-4
    assert np.all(np.isfinite(C))


def test_conv_fp32x_l8192(W):
    """Full 8192/16/8192 sum on 8192 GL angles; vs the FP64 kernel (every 16th angle) and the oracle."""
    L, MB, MS, beta, a, b = I.make_config("conv_fp32x_l8192")
    beta_d, a_d, b_d = _cuda(beta), _cuda(a), _cuda(b)
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    C32 = W.wigner_conv_sum(beta_d, a_d, b_d, form="fp32x", counters=cnt)
    W.check_device_status()
    assert int(cnt[0]) == I.n_elements(L, MB, MS, beta.size)
    sel = np.arange(0, beta.size, 16)
    C64 = W.wigner_conv_sum(_cuda(beta[sel]), a_d, b_d, form="fp64")
    W.check_device_status()
    sub = C32[:, :, torch.from_numpy(sel).cuda()]
    rel = float((torch.linalg.vector_norm(sub - C64) / torch.linalg.vector_norm(C64)).item())
    assert rel <= 1e-4, rel
    assert bool(torch.isfinite(torch.view_as_real(C32)).all())
    rng = np.random.default_rng(0)
    n = 200
    idx = np.stack([rng.integers(0, MB + 1, n), rng.integers(0, MS + 1, n), rng.integers(0, beta.size, n)], 1)
    idx[:4] = [[0, 0, 0], [MB, MS, beta.size - 1], [0, 0, beta.size - 1], [MB, 0, 0]]
    ti = [torch.from_numpy(idx[:, k]).cuda() for k in range(3)]
    got = C32[ti[0], ti[1], ti[2]].cpu().numpy()
    ref = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    assert _rel_l2(got, ref) <= 1e-4


def test_conv_fp32x_size_limits_sampled(W):
    """The FP32 form at the longest chains (l_max = 32767) and at chains starting at
    m_b = m_sky ~ 2000 (the fastest growth in the four steps between rescales)."""
    L, MB, MS = W.WG_LMAX, 2, 300
    beta = np.array([0.05, 1.0, math.pi / 2, math.pi - 0.05])
    a = I.sky_alm(L, MS, 12)
    b = I.beam_blm(L, MB, fwhm=0.001)
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form="fp32x").cpu().numpy()
    W.check_device_status()
    rng = np.random.default_rng(1)
    idx = np.stack([rng.integers(0, MB + 1, 48), rng.integers(0, MS + 1, 48), rng.integers(0, beta.size, 48)], 1)
    ref = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    assert _rel_l2(C[idx[:, 0], idx[:, 1], idx[:, 2]], ref) <= 1e-4

    L, MB, MS = 2100, 2000, 2000
    beta = np.array([0.02, 0.7, math.pi / 2, 2.5, math.pi - 0.02])
    a = I.sky_alm(L, MS, 13)
    rng = np.random.default_rng(14)
    b = rng.standard_normal((L + 1, MB + 1)) + 1j * rng.standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form="fp32x").cpu().numpy()
    W.check_device_status()
    assert np.all(np.isfinite(C))
    idx = np.array([[2000, 2000, j] for j in range(5)] + [[1999, 2000, 0], [2000, 1999, 4], [1500, 1800, 1],
                                                          [1800, 1500, 3], [0, 2000, 2], [2000, 0, 1]])
    ref = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    assert _rel_l2(C[idx[:, 0], idx[:, 1], idx[:, 2]], ref) <= 1e-4


def test_conv_fp32x_columns_from_l0_8192(W):
    """Away from the poles the FP32 form runs the normalised recursion, except for
    columns starting at l0 >= 8192 (difference form, x^2 derived from cos(beta)); a sum
    whose columns straddle that limit, sampled against the oracle."""
    L, MB, MS = 8250, 0, 8250
    beta = np.array([1.45, 1.52, 1.6, 1.68])  # near pi/2: the orders m_sky ~ 8200 reach their turning point
    a = I.sky_alm(L, MS, 15)
    b = I.beam_blm(L, MB, fwhm=0.0005)
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form="fp32x").cpu().numpy()
    W.check_device_status()
    assert np.all(np.isfinite(C))
    ms = [0, 100, 4000, 8100, 8191, 8192, 8193, 8200, 8249, 8250]
    idx = np.array([[0, m, j] for m in ms for j in range(beta.size)])
    ref = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    got = C[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert _rel_l2(got, ref) <= 1e-4
    hi = idx[:, 1] >= 8192  # the difference-form columns on their own
    assert _rel_l2(got[hi], ref[hi]) <= 1e-4
