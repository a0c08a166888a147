"""GPU parity of the l_min cut (Sec. 4.2.1, Eq. lmin) against the oracle's cut sum, through
the C-ABI: positive orders and every sky order, both FP64 forms, offsets from 0 (the cut
at the turning point, where the cut terms matter most) to one that cuts nothing.  Bar:
1e-11 absolute, elementwise; chains cut whole are exactly 0."""
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


def mirror_grid(n):
    g = I.beta_gauss_legendre(n)[0]
    h = n // 2
    out = g.copy()
    out[n - h:] = math.pi - g[:h][::-1]
    if n % 2:
        out[h] = math.pi / 2
    return out


@pytest.mark.parametrize("form", ["fp64", "fp64s"])
@pytest.mark.parametrize("offset", [0.0, 5.0, 15.0, 30.0])
@pytest.mark.parametrize("L,MB,MS,NB,grid", [(300, 4, 300, 513, "gl"), (150, 8, 60, 257, "poles")])
def test_lmin_matches_oracle(W, form, offset, L, MB, MS, NB, grid):
    if grid == "gl":
        beta = I.beta_gauss_legendre(NB)[0]
    else:
        beta = I.beta_uniform(NB, 0.0, math.pi, 9)
        beta[:4] = [0.0, math.pi, 1e-7, math.pi - 1e-6]
    a = I.sky_alm(L, MS, 21)
    b = I.beam_blm(L, MB, fwhm=0.05) + 0.01j
    C = W.wigner_conv_sum_lmin(_cuda(beta), _cuda(a), _cuda(b), offset, form=form).cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum(L, MB, MS, beta, a, b, offset=offset)
    assert np.max(np.abs(C - ref)) <= TOL
    cut = np.array([[[O.l_first(L, mb, ms, bt, offset) > L for bt in beta] for ms in range(MS + 1)]
                    for mb in range(MB + 1)])
    assert np.all(C[cut] == 0)


@pytest.mark.parametrize("form", ["fp64", "fp64s"])
@pytest.mark.parametrize("offset", [0.0, 10.0, 40.0])
def test_lmin_full_matches_oracle(W, form, offset):
    L, MB, MS, NB = 200, 3, 200, 301
    beta = mirror_grid(NB)
    a, b = I.sky_alm(L, MS, 22), I.beam_blm(L, MB, fwhm=0.05)
    C = W.wigner_conv_sum_lmin(_cuda(beta), _cuda(a), _cuda(b), offset, form=form, full=True).cpu().numpy()
    W.check_device_status()
    assert np.max(np.abs(C - O.conv_sum_full(L, MB, MS, beta, a, b, offset=offset))) <= TOL


@pytest.mark.parametrize("form", ["fp64", "fp64s"])
def test_lmin_large_offset_is_the_sum(W, form):
    """An offset that cuts nothing gives wigner_conv_sum's result bit for bit."""
    L, MB, MS, NB = 260, 5, 260, 400
    beta = _cuda(I.beta_gauss_legendre(NB)[0])
    a, b = _cuda(I.sky_alm(L, MS, 23)), _cuda(I.beam_blm(L, MB))
    c1 = W.wigner_conv_sum(beta, a, b, form=form)
    c2 = W.wigner_conv_sum_lmin(beta, a, b, float(MB + MS), form=form)
    assert torch.equal(c1, c2)


def test_lmin_skips_work(W):
    """Cut chains are not evaluated: at offset 0 about 17 % of the elements belong to warps
    (64 consecutive angles) whose chains are all cut, and the counter drops by that."""
    L, MB, MS, NB = 1000, 4, 1000, 1024
    beta = I.beta_gauss_legendre(NB)[0]
    a, b = I.sky_alm(L, MS, 24), I.beam_blm(L, MB)
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    W.wigner_conv_sum_lmin(_cuda(beta), _cuda(a), _cuda(b), 0.0, counters=cnt)
    full = I.n_elements(L, MB, MS, NB)
    assert int(cnt[0]) < 0.88 * full


def test_lmin_l4096_sampled(W):
    """The L=4096 workload with the paper's offset L/20 and with 15, sampled."""
    L, MB, MS, beta, a, b = I.make_config("conv_fp64_l4096")
    rng = np.random.default_rng(6)
    n = 200
    idx = np.stack([rng.integers(0, MB + 1, n), rng.integers(0, MS + 1, n), rng.integers(0, beta.size, n)], 1)
    idx[:3] = [[0, 3000, 100], [8, 100, 5], [2, 4096, 2047]]
    ti = [torch.from_numpy(idx[:, q]).cuda() for q in range(3)]
    for offset in (L / 20, 15.0):
        C = W.wigner_conv_sum_lmin(_cuda(beta), _cuda(a), _cuda(b), offset)
        W.check_device_status()
        got = C[ti[0], ti[1], ti[2]].cpu().numpy()
        ref = O.conv_sum_full_sampled(L, MB, MS, beta, a, b, idx, offset=offset)
        assert np.max(np.abs(got - ref)) <= TOL
        del C
