"""GPU parity of the sum over every sky order (the C_{m_b m_sky}(beta), -ms_max <= m_sky <=
ms_max, of the conviqt data cube, Sec. 4.1 Eq. conviqt).

The kernel takes the negative orders from the positive chains through the pi - beta
identity on a mirror-symmetric grid; the oracle runs a chain of its own for every
negative order (general edge seeds), so the two routes are independent.  Bar: 1e-11
absolute (FP64 path), elementwise.
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


def mirror_grid(n):
    """Gauss-Legendre angles made exactly mirror-symmetric: the upper half is pi minus the lower."""
    g = I.beta_gauss_legendre(n)[0]
    h = n // 2
    out = g.copy()
    out[n - h:] = math.pi - g[:h][::-1]
    if n % 2:
        out[h] = math.pi / 2
    return out


@pytest.mark.parametrize("form", ["fp64", "fp64s"])
@pytest.mark.parametrize("L,MB,MS,NB", [(150, 4, 150, 300), (90, 8, 40, 301), (1, 1, 1, 2), (0, 0, 0, 1),
                                        (300, 2, 300, 513)])
def test_full_matches_oracle(W, form, L, MB, MS, NB):
    beta = mirror_grid(NB)
    a = I.sky_alm(L, MS, 31)
    b = I.beam_blm(L, MB, fwhm=0.05) + 0.02j * np.random.default_rng(32).standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    C = W.wigner_conv_sum_full(_cuda(beta), _cuda(a), _cuda(b), form=form).cpu().numpy()
    W.check_device_status()
    ref = O.conv_sum_full(L, MB, MS, beta, a, b)
    assert np.max(np.abs(C - ref)) <= TOL
    # the non-negative orders are exactly the ones wigner_conv_sum computes
    Cp = W.wigner_conv_sum(_cuda(beta), _cuda(a), _cuda(b), form=form).cpu().numpy()
    assert np.array_equal(C[:, MS:, :], Cp)


def test_full_l4096_sampled(W):
    """The L=4096 workload over every sky order (2048 mirror-symmetric GL angles), sampled."""
    L, MB, MS, _, a, b = I.make_config("conv_fp64_l4096")
    beta = mirror_grid(2048)
    C = W.wigner_conv_sum_full(_cuda(beta), _cuda(a), _cuda(b))
    W.check_device_status()
    rng = np.random.default_rng(4)
    n = 300
    idx = np.stack([rng.integers(0, MB + 1, n), rng.integers(-MS, MS + 1, n), rng.integers(0, beta.size, n)], 1)
    idx[:6] = [[0, -MS, 0], [MB, -MS, beta.size - 1], [MB, -1, 0], [0, -1, beta.size - 1], [3, -2000, 1024],
               [8, MS, 7]]
    ti = [torch.from_numpy(idx[:, 0]).cuda(), torch.from_numpy(idx[:, 1] + MS).cuda(),
          torch.from_numpy(idx[:, 2]).cuda()]
    got = C[ti[0], ti[1], ti[2]].cpu().numpy()
    ref = O.conv_sum_full_sampled(L, MB, MS, beta, a, b, idx)
    assert np.max(np.abs(got - ref)) <= TOL
    assert bool(torch.isfinite(torch.view_as_real(C)).all())


def test_full_rejects_asymmetric_grid(W):
    """A grid that is not mirror-symmetric: the negative orders are NaN and the device status says so."""
    L, MB, MS, NB = 30, 2, 30, 40
    beta = I.beta_uniform(NB, 0.05, math.pi - 0.05, 33)
    a, b = I.sky_alm(L, MS, 34), I.beam_blm(L, MB, fwhm=0.1)
    C = W.wigner_conv_sum_full(_cuda(beta), _cuda(a), _cuda(b)).cpu().numpy()
    with pytest.raises(W.WignerError):
        W.check_device_status()
    assert np.all(np.isnan(C[:, :MS, :]))
    assert np.max(np.abs(C[:, MS:, :] - O.conv_sum(L, MB, MS, beta, a, b))) <= TOL
    W.check_device_status()  # cleared


def test_full_fp32x_unsupported(W):
    beta = mirror_grid(8)
    a, b = I.sky_alm(10, 10, 1), I.beam_blm(10, 2)
    with pytest.raises(W.WignerError):
        W.wigner_conv_sum_full(_cuda(beta), _cuda(a), _cuda(b), form="fp32x")


def cube_reference(Cf, n_alpha, n_gamma, js=None, ps=None, qs=None):
    """Eq. conviqt written out: sum over m_b in [-M, M], m_sky in [-S, S] of
    e^{-i m_b alpha} e^{-i m_sky gamma} C_{m_b m_sky}(beta), C_{-m_b,-m} = conj(C_{m_b m}).
    Cf: (M+1, 2S+1, N).  Returns the complex sums (their imaginary parts vanish for real fields)."""
    M, S = Cf.shape[0] - 1, (Cf.shape[1] - 1) // 2
    js = range(Cf.shape[2]) if js is None else js
    ps = np.arange(n_alpha) if ps is None else np.asarray(ps)
    qs = np.arange(n_gamma) if qs is None else np.asarray(qs)
    mbs, mss = np.arange(-M, M + 1), np.arange(-S, S + 1)
    Ea = np.exp(-1j * np.outer(2 * np.pi * ps / n_alpha, mbs))
    Eg = np.exp(-1j * np.outer(2 * np.pi * qs / n_gamma, mss))
    out = []
    for j in js:
        full = np.empty((2 * M + 1, 2 * S + 1), dtype=np.complex128)
        full[M:, :] = Cf[:, :, j]
        full[:M, :] = np.conj(Cf[1:, ::-1, j])[::-1]  # C_{-m_b, m} = conj(C_{m_b, -m})
        out.append(Ea @ full @ Eg.T)
    return np.array(out)


@pytest.mark.parametrize("n_alpha,n_gamma", [(None, None), (11, 90), (8, 81)])
def test_data_cube_matches_definition(W, n_alpha, n_gamma):
    L, MB, MS, NB = 40, 3, 40, 12
    beta = mirror_grid(NB)
    a, b = I.sky_alm(L, MS, 41), I.beam_blm(L, MB, fwhm=0.1)
    Cg = W.wigner_conv_sum_full(_cuda(beta), _cuda(a), _cuda(b))
    cube = W.wigner_data_cube(Cg, n_alpha, n_gamma)
    W.check_device_status()
    na, ng = cube.shape[1], cube.shape[2]
    assert na >= 2 * MB + 1 and ng >= 2 * MS + 1
    ref = cube_reference(O.conv_sum_full(L, MB, MS, beta, a, b), na, ng)
    scale = float(np.max(np.abs(ref)))
    assert float(np.max(np.abs(ref.imag))) <= 1e-12 * scale  # a real sky and beam give a real cube
    assert float(np.max(np.abs(cube.cpu().numpy() - ref.real))) <= 1e-12 * scale


def test_data_cube_l4096_sampled(W):
    """The L=4096 workload's cube (2048 mirror-symmetric angles, 18 x 8232 per angle) at two
    angles, every alpha and 64 gamma, against the definition on the oracle's C."""
    L, MB, MS, _, a, b = I.make_config("conv_fp64_l4096")
    beta = mirror_grid(2048)
    Cg = W.wigner_conv_sum_full(_cuda(beta), _cuda(a), _cuda(b))
    cube = W.wigner_data_cube(Cg)
    W.check_device_status()
    rng = np.random.default_rng(9)
    qs = rng.integers(0, cube.shape[2], 64)
    for j in (3, 1500):
        Co = O.conv_sum_full(L, MB, MS, beta[[j]], a, b)
        ref = cube_reference(Co, cube.shape[1], cube.shape[2], qs=qs)[0]
        got = cube[j].cpu().numpy()[:, qs]
        assert float(np.max(np.abs(got - ref.real))) <= 1e-10 * max(1.0, float(np.max(np.abs(ref))))


def test_data_cube_rejects_aliasing(W):
    Cg = torch.zeros((3, 21, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(W.WignerError):
        W.wigner_data_cube(Cg, 4, 30)   # n_alpha < 2 mb_max + 1
    with pytest.raises(W.WignerError):
        W.wigner_data_cube(Cg, 8, 20)   # n_gamma < 2 ms_max + 1
