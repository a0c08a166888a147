"""GPU parity of the FP64 d-table and fused-sum kernels against the CPU oracle.

Tolerance: 1e-11 absolute, elementwise (FP64 path bar).  Inputs are the seeded
workloads of paper_1002_1050_gb300.inputs; small cases span several l-tiles,
several angle chunks and ragged tails; the full 4096/8/4096/2048 sum is checked on
sampled outputs that the oracle computes one by one.
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import wigner
    wigner.load()
    return wigner


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_dtable_l256_full(W):
    """The 256/4/256/64-angle d-table, every element."""
    L, MB, MS, beta, _, _ = I.make_config("dtable_l256")
    d = W.wigner_d_table(_cuda(beta), L, MB, MS).cpu().numpy()
    W.check_device_status()
    ref = O.d_table(L, MB, MS, beta)
    err = np.max(np.abs(d - ref))
    assert err <= TOL, err


@pytest.mark.parametrize("L,MB,MS,NB", [(0, 0, 0, 1), (1, 1, 1, 3), (2, 2, 2, 5), (37, 5, 37, 71),
                                        (300, 12, 150, 130)])
def test_dtable_small_ragged(W, L, MB, MS, NB):
    beta = np.concatenate([[0.0, math.pi], I.beta_uniform(max(NB - 2, 0), 1e-4, math.pi - 1e-4, 3)])[:NB]
    d = W.wigner_d_table(_cuda(beta), L, MB, MS).cpu().numpy()
    W.check_device_status()
    ref = O.d_table(L, MB, MS, beta)
    assert np.max(np.abs(d - ref)) <= TOL


def test_dtable_long_columns_and_poles(W):
    """Columns past l0 = 1024 and angles next to the poles, where the seed's logarithm is
    large, against the oracle's chains at the FP64 bar; also more angle chunks (40
    angles: a full and a ragged 32-angle chunk).  (Near the poles Eq. lrec's two roots
    merge and two double-precision evaluations of a chain drift apart like l^2 times
    the rounding unit: about 1e-11 at l = 1500, 6e-12 at l = 1100.)"""
    L, MB, MS = 1100, 16, 1100
    beta = np.concatenate([[0.0, 1e-4, 2e-3, math.pi / 2, math.pi - 2e-3, math.pi - 1e-4, math.pi],
                           I.beta_uniform(33, 1e-3, math.pi - 1e-3, 8)])
    d = W.wigner_d_table(_cuda(beta), L, MB, MS)
    W.check_device_status()
    for mb, ms in [(0, 0), (16, 16), (3, 700), (16, 1030), (5, 1050), (16, 1099), (0, 1100), (11, 1024),
                   (7, 1025)]:
        ref = O.d_column(L, mb, ms, beta)
        got = d[mb, ms].cpu().numpy()
        assert float(np.max(np.abs(got - ref))) <= TOL, (mb, ms)
    del d
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", ["fp64", "fp32x"])
@pytest.mark.parametrize("L,MB,MS,NB", [(256, 4, 256, 64), (300, 12, 150, 45), (40, 40, 7, 33), (5, 5, 5, 2),
                                        (0, 0, 0, 3)])
def test_dtable_every_row_written(W, form, L, MB, MS, NB):
    """The output starts as NaN: every element, the zeros for l < l0 included, is written by
    the kernels (the FP64 kernel writes a column's zero rows from another column's item)."""
    beta = I.beta_uniform(NB, 1e-3, math.pi - 1e-3, 5)
    out = torch.full((MB + 1, MS + 1, L + 1, NB), float("nan"), dtype=torch.float64, device="cuda")
    d = W.wigner_d_table(_cuda(beta), L, MB, MS, form=form, out=out).cpu().numpy()
    W.check_device_status()
    assert not np.isnan(d).any()
    ref = O.d_table(L, MB, MS, beta)
    l0 = np.maximum(np.arange(MB + 1)[:, None], np.arange(MS + 1)[None, :])
    zero = np.arange(L + 1)[None, None, :] < l0[:, :, None]
    assert np.all(d[zero] == 0.0)
    assert np.max(np.abs(d - ref)) <= (TOL if form == "fp64" else 2e-4)


def test_dtable_counters(W):
    L, MB, MS, beta, _, _ = I.make_config("dtable_l256")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    W.wigner_d_table(_cuda(beta), L, MB, MS, counters=cnt)
    assert int(cnt[0]) == I.n_elements(L, MB, MS, beta.size) == 10_607_680


def _complex_beam(L, MB, seed):
    rng = np.random.default_rng(seed)
    b = I.beam_blm(L, MB, fwhm=0.05) + 0.05j * rng.standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    return np.ascontiguousarray(b)


FORMS = ["fp64", "fp64s"]  # all-double kernel; split-pipe kernel (FP64 recursion, float-float sum)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,MB,MS,NB,grid", [(64, 4, 64, 300, "gl"), (200, 8, 120, 513, "uniform"),
                                             (129, 16, 129, 31, "gl"), (1, 1, 1, 2, "uniform"),
                                             (700, 3, 700, 40, "uniform")])
def test_conv_small_full(W, L, MB, MS, NB, grid, form):
    beta = I.beta_gauss_legendre(NB)[0] if grid == "gl" else I.beta_uniform(NB, 1e-3, math.pi - 1e-3, 11)
    a = I.sky_alm(L, MS, 5)
    b = _complex_beam(L, MB, 6)
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form=form).cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum(L, MB, MS, beta, a, b)
    assert np.max(np.abs(C - ref)) <= TOL


@pytest.mark.parametrize("form", FORMS)
def test_conv_endpoints_and_bad_angle(W, form):
    L, MB, MS = 40, 3, 40
    a = I.sky_alm(L, MS, 1)
    b = _complex_beam(L, MB, 2)
    beta = np.array([0.0, math.pi, 0.5, 1.0])
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form=form).cpu().numpy()
    W.check_device_status()
    assert np.max(np.abs(C - O.conv_sum(L, MB, MS, beta, a, b))) <= TOL
    # an angle outside [0, pi]: its outputs are NaN and the status word reports it
    beta_bad = np.array([0.5, -0.1, 4.0, 1.0])
    C = W.wigner_conv_sum(_cuda(beta_bad), _cuda(a), _cuda(b), form=form).cpu().numpy()
    assert W.wigner_device_status() == -1
    assert np.all(np.isnan(C[:, :, 1])) and np.all(np.isnan(C[:, :, 2]))
    assert np.max(np.abs(C[:, :, [0, 3]] - O.conv_sum(L, MB, MS, beta_bad[[0, 3]], a, b))) <= TOL
    assert W.wigner_device_status() == 0  # cleared


@pytest.mark.parametrize("form", FORMS)
def test_conv_l4096_sampled(W, form):
    """Full-size fused FP64 sum (L=4096, m_b<=8, m_sky<=4096, 2048 GL angles), sampled outputs."""
    L, MB, MS, beta, a, b = I.make_config("conv_fp64_l4096")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form=form, counters=cnt)
    W.check_device_status()
    assert int(cnt[0]) == I.n_elements(L, MB, MS, beta.size)
    rng = np.random.default_rng(0)
    n = 400
    idx = np.stack([rng.integers(0, MB + 1, n), rng.integers(0, MS + 1, n), rng.integers(0, beta.size, n)], 1)
    # always include the extreme columns and angles
    idx[:4] = [[0, 0, 0], [MB, MS, beta.size - 1], [0, MS, 0], [MB, 0, beta.size - 1]]
    got = C.cpu().numpy()[idx[:, 0], idx[:, 1], idx[:, 2]]
    ref = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    assert np.max(np.abs(got - ref)) <= TOL
    assert np.all(np.isfinite(C.cpu().numpy()))


def _random_beam(L, MB, seed):
    """Complex beam weights of order one for every m_b <= min(l, MB) (a stress input whose
    high-m_b columns do not vanish, unlike the Gaussian beam's)."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((L + 1, MB + 1)) + 1j * rng.standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    return b / np.sqrt(L + 1.0)


def _sample_idx(MB, MS, NB, n, seed, extra):
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, MB + 1, n), rng.integers(0, MS + 1, n), rng.integers(0, NB, n)], 1)
    idx[:len(extra)] = extra
    return idx


@pytest.mark.parametrize("form", FORMS)
def test_conv_longest_chains_sampled(W, form):
    """The longest chains the library accepts (l_max = WG_LMAX = 32767), 301 sky orders, a
    near-pole angle; sampled outputs against the oracle."""
    L, MB, MS = W.WG_LMAX, 2, 300
    beta = np.array([0.05, 1.0, math.pi / 2, math.pi - 0.05])
    a = I.sky_alm(L, MS, 12)
    b = I.beam_blm(L, MB, fwhm=0.001)
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form=form).cpu().numpy()
    W.check_device_status()
    idx = _sample_idx(MB, MS, beta.size, 48, 1,
                      [[0, 0, 0], [2, 300, 0], [0, 0, 3], [2, 300, 3], [1, 150, 2], [2, 2, 1]])
    ref = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    assert np.max(np.abs(C[idx[:, 0], idx[:, 1], idx[:, 2]] - ref)) <= TOL
    assert np.all(np.isfinite(C))


@pytest.mark.parametrize("form", FORMS)
def test_conv_large_equal_orders_sampled(W, form):
    """Chains starting at l0 = m_b = m_sky ~ 2000 (the largest coefficients F0 ~ l0 of the
    first steps) and the whole 2001 x 2001 column range; sampled outputs."""
    L, MB, MS = 2100, 2000, 2000
    beta = np.array([0.02, 0.7, math.pi / 2, 2.5, math.pi - 0.02])
    a = I.sky_alm(L, MS, 13)
    b = _random_beam(L, MB, 14)
    C = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form=form).cpu().numpy()
    W.check_device_status()
    extra = [[2000, 2000, j] for j in range(5)] + [[1999, 2000, 0], [2000, 1999, 4], [0, 2000, 2], [2000, 0, 1]]
    idx = _sample_idx(MB, MS, beta.size, 60, 2, extra)
    ref = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    assert np.max(np.abs(C[idx[:, 0], idx[:, 1], idx[:, 2]] - ref)) <= TOL
    assert np.all(np.isfinite(C))
