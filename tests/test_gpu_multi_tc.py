"""GPU parity of the tensor-core many-sky sum (wigner_conv_sum_multi_tc: split-bf16 slices,
tcgen05.mma, float-float fold) against the CPU oracle, through the C-ABI.

The oracle runs each sky's Eq. convdef sum on its own (conv_sum_multi).  Bar: 1e-11
absolute, elementwise (the FP64 path's bar), on ragged sizes (angle counts that are not
multiples of the 128-angle CTA, chain lengths that end inside a 32-order tile and span
several 256-order segments, sky counts that are not multiples of the 32 per launch
column group), real and complex beams, the poles, degenerate sizes, and the L = 4096
workload with 32 Monte-Carlo skies on sampled outputs."""
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


def _complex_beam(L, MB, seed, fwhm=0.05):
    rng = np.random.default_rng(seed)
    b = I.beam_blm(L, MB, fwhm=fwhm) + 0.1j * rng.standard_normal((L + 1, MB + 1)) / np.sqrt(1.0 + np.arange(L + 1))[:, None]
    b[:, 0] = b[:, 0].real  # one order with a real beam (its imaginary pass is skipped)
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    return np.ascontiguousarray(b)


@pytest.mark.parametrize("n_col", [1, 8, 16, 33])
@pytest.mark.parametrize("L,MB,MS,NB", [(300, 4, 300, 513), (130, 8, 40, 257), (63, 2, 63, 129)])
def test_tc_real_beam(W, n_col, L, MB, MS, NB):
    beta = I.beta_gauss_legendre(NB)[0]
    a = I.mc_skies(L, MS, n_col, 50)
    b = I.beam_blm(L, MB, fwhm=0.05)
    C = W.wigner_conv_sum_multi_tc(_cuda(beta), _cuda(a), _cuda(b)).cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum_multi(L, MB, MS, beta, a, b)
    err = float(np.max(np.abs(C - ref)))
    assert err <= TOL, err


@pytest.mark.parametrize("n_col", [16, 64])
def test_tc_complex_beam_ragged(W, n_col):
    L, MB, MS, NB = 211, 5, 190, 301
    beta = I.beta_uniform(NB, 0.0, math.pi, 9)
    beta[:4] = [0.0, math.pi, 1e-7, math.pi - 1e-7]  # poles and near-pole angles
    a = I.mc_skies(L, MS, n_col, 7)
    b = _complex_beam(L, MB, 3)
    C = W.wigner_conv_sum_multi_tc(_cuda(beta), _cuda(a), _cuda(b)).cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum_multi(L, MB, MS, beta, a, b)
    err = float(np.max(np.abs(C - ref)))
    assert err <= TOL, err


@pytest.mark.parametrize("L,MB,MS,NB,n_col", [(0, 0, 0, 1, 2), (1, 1, 1, 2, 3), (5, 5, 5, 1, 9), (31, 3, 31, 128, 8),
                                              (32, 3, 32, 130, 8), (600, 2, 20, 40, 8)])
def test_tc_degenerate_sizes(W, L, MB, MS, NB, n_col):
    beta = I.beta_uniform(NB, 0.1, 3.0, 2)
    a = I.mc_skies(L, MS, n_col, 3)
    b = _complex_beam(L, MB, 4, fwhm=0.3)
    C = W.wigner_conv_sum_multi_tc(_cuda(beta), _cuda(a), _cuda(b)).cpu().numpy()
    W.check_device_status()
    err = float(np.max(np.abs(C - O.conv_sum_multi(L, MB, MS, beta, a, b))))
    assert err <= TOL, err


def test_tc_routing_and_counters(W):
    """wigner_conv_sum_multi with a shared beam and >= 8 skies takes the tensor-core path
    (bitwise the same result); the counters count every chain once."""
    L, MB, MS, NB = 150, 4, 150, 200
    beta = _cuda(I.beta_gauss_legendre(NB)[0])
    a, b = _cuda(I.mc_skies(L, MS, 8, 4)), _cuda(I.beam_blm(L, MB))
    c = torch.zeros(2, dtype=torch.int64, device="cuda")
    C1 = W.wigner_conv_sum_multi(beta, a, b)
    C2 = W.wigner_conv_sum_multi_tc(beta, a, b, counters=c)
    W.check_device_status()
    assert torch.equal(C1, C2)
    assert int(c[0]) == int(c[1]) == I.n_elements(L, MB, MS, NB)


def test_tc_bad_angle_and_timeout(W):
    L, MB, MS, NB = 120, 3, 120, 150
    beta_h = I.beta_gauss_legendre(NB)[0]
    beta_h[7] = -0.5
    beta = _cuda(beta_h)
    a, b = I.mc_skies(L, MS, 8, 5), _complex_beam(L, MB, 5)
    ta, tb = _cuda(a), _cuda(b)
    C = W.wigner_conv_sum_multi_tc(beta, ta, tb).cpu().numpy()
    assert W.wigner_device_status() == -1  # WG_ERR_ARG: the angle outside [0, pi]
    assert np.all(np.isnan(C[:, :, :, 7])) and not np.isnan(np.delete(C, 7, axis=3)).any()
    beta_h[7] = 1.0
    beta = _cuda(beta_h)
    old = W.debug_set_wait_tries(0)
    try:
        C = W.wigner_conv_sum_multi_tc(beta, ta, tb)
        rc = W.wigner_device_status()
    finally:
        W.debug_set_wait_tries(old)
    assert rc == -4  # WG_ERR_TIMEOUT: every bounded wait gave up, the context survives
    assert bool(torch.isnan(C).all())
    C = W.wigner_conv_sum_multi_tc(beta, ta, tb).cpu().numpy()
    assert W.wigner_device_status() == 0
    assert float(np.max(np.abs(C - O.conv_sum_multi(L, MB, MS, beta_h, a, b)))) <= TOL


def test_tc_l4096_32_skies_sampled(W):
    """32 Monte-Carlo skies on the L=4096 workload (one launch column group), sampled
    against the oracle per sky."""
    L, MB, MS, beta, _, b = I.make_config("conv_fp64_l4096")
    K = 32
    a = I.mc_skies(L, MS, K, 70)
    C = W.wigner_conv_sum_multi_tc(_cuda(beta), _cuda(a), _cuda(b))
    W.check_device_status()
    rng = np.random.default_rng(6)
    n = 60
    idx = np.stack([rng.integers(0, MB + 1, n), rng.integers(0, MS + 1, n), rng.integers(0, beta.size, n)], 1)
    idx[:4] = [[0, 0, 0], [MB, MS, beta.size - 1], [8, 4000, 1024], [0, 1, 1]]
    ti = [torch.from_numpy(idx[:, q]).cuda() for q in range(3)]
    worst = 0.0
    for k in range(K):
        got = C[k][ti[0], ti[1], ti[2]].cpu().numpy()
        ref = O.conv_sum_sampled(L, MB, MS, beta, a[k], b, idx)
        worst = max(worst, float(np.max(np.abs(got - ref))))
    assert worst <= TOL, worst
    assert bool(torch.isfinite(torch.view_as_real(C)).all())
    del C
    torch.cuda.empty_cache()
