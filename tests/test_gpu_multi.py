"""GPU parity of the several-column sum (Eq. convdef for Monte-Carlo skies sharing a beam
and for the polarised pairs of the footnote of Sec. 4.1), through the C-ABI.

The kernel runs one recursion per pass of up to four columns; the oracle runs each
column's sum on its own.  Bar: 1e-11 absolute (FP64 forms), elementwise."""
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


@pytest.mark.parametrize("form", ["fp64", "fp64s"])
@pytest.mark.parametrize("n_col", [1, 3, 4, 5, 9])
@pytest.mark.parametrize("L,MB,MS,NB", [(300, 4, 300, 513), (130, 8, 40, 257)])
def test_mc_shared_beam(W, form, n_col, L, MB, MS, NB):
    beta = I.beta_gauss_legendre(NB)[0]
    a = I.mc_skies(L, MS, n_col, 50)
    b = I.beam_blm(L, MB, fwhm=0.05)
    C = W.wigner_conv_sum_multi(_cuda(beta), _cuda(a), _cuda(b), form=form).cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum_multi(L, MB, MS, beta, a, b)
    assert np.max(np.abs(C - ref)) <= TOL


@pytest.mark.parametrize("form", ["fp64", "fp64s"])
@pytest.mark.parametrize("sum_cols", [False, True])
def test_polarised_pairs(W, form, sum_cols):
    L, MB, MS, NB = 257, 4, 200, 300
    beta = I.beta_uniform(NB, 0.0, math.pi, 7)
    beta[:3] = [0.0, math.pi, 1e-7]  # poles and a near-pole angle
    a, b = I.polarised_columns(L, MB, MS, 60)
    C = W.wigner_conv_sum_multi(_cuda(beta), _cuda(a), _cuda(b), form=form, sum_cols=sum_cols).cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum_multi(L, MB, MS, beta, a, b, sum_cols=sum_cols)
    assert C.shape == ref.shape
    assert np.max(np.abs(C - ref)) <= TOL


@pytest.mark.parametrize("L,MB,MS,NB,n_col", [(0, 0, 0, 1, 2), (1, 1, 1, 2, 3), (5, 5, 5, 1, 1)])
def test_multi_degenerate_sizes(W, L, MB, MS, NB, n_col):
    beta = I.beta_uniform(NB, 0.1, 3.0, 2)
    a = I.mc_skies(L, MS, n_col, 3)
    b = np.stack([I.beam_blm(L, MB, fwhm=0.3)] * n_col) * (1 + 0.5j)
    C = W.wigner_conv_sum_multi(_cuda(beta), _cuda(a), _cuda(b)).cpu().numpy()
    W.check_device_status()
    assert np.max(np.abs(C - O.conv_sum_multi(L, MB, MS, beta, a, b))) <= TOL


def test_multi_empty(W):
    beta = torch.zeros(0, dtype=torch.float64, device="cuda")
    a = _cuda(I.mc_skies(10, 10, 2, 1))
    b = _cuda(I.beam_blm(10, 2))
    assert W.wigner_conv_sum_multi(beta, a, b).shape == (2, 3, 11, 0)
    z = W.wigner_conv_sum_multi(_cuda(I.beta_uniform(5, 0.1, 3.0, 1)), a[:0], b, sum_cols=True)
    assert z.shape == (3, 11, 5) and not bool(z.abs().any())  # no columns: zeros


def test_multi_counters_count_the_chains_once(W):
    L, MB, MS, NB = 200, 4, 200, 100
    beta = _cuda(I.beta_gauss_legendre(NB)[0])
    a, b = _cuda(I.mc_skies(L, MS, 6, 4)), _cuda(I.beam_blm(L, MB))
    c1 = torch.zeros(2, dtype=torch.int64, device="cuda")
    c6 = torch.zeros(2, dtype=torch.int64, device="cuda")
    W.wigner_conv_sum(beta, a[0], b, counters=c1)
    W.wigner_conv_sum_multi(beta, a, b, counters=c6)
    assert int(c6[0]) == int(c1[0]) == I.n_elements(L, MB, MS, NB)


def test_multi_fp32x_unsupported(W):
    beta = _cuda(I.beta_uniform(8, 0.1, 3.0, 1))
    with pytest.raises(W.WignerError):
        W.wigner_conv_sum_multi(beta, _cuda(I.mc_skies(10, 10, 2, 1)), _cuda(I.beam_blm(10, 2)), form="fp32x")


def test_mc_l4096_sampled(W):
    """Four skies on the L=4096 workload (one pass), sampled against the oracle per column."""
    L, MB, MS, beta, _, b = I.make_config("conv_fp64_l4096")
    a = I.mc_skies(L, MS, 4, 70)
    C = W.wigner_conv_sum_multi(_cuda(beta), _cuda(a), _cuda(b))
    W.check_device_status()
    rng = np.random.default_rng(5)
    n = 200
    idx = np.stack([rng.integers(0, MB + 1, n), rng.integers(0, MS + 1, n), rng.integers(0, beta.size, n)], 1)
    idx[:4] = [[0, 0, 0], [MB, MS, beta.size - 1], [8, 4000, 1024], [0, 1, 1]]
    ti = [torch.from_numpy(idx[:, q]).cuda() for q in range(3)]
    for k in range(4):
        got = C[k][ti[0], ti[1], ti[2]].cpu().numpy()
        ref = O.conv_sum_sampled(L, MB, MS, beta, a[k], b, idx)
        assert np.max(np.abs(got - ref)) <= TOL
    assert bool(torch.isfinite(torch.view_as_real(C)).all())
