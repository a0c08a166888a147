"""GPU parity of the full-matrix evaluator (Sec. 3.1: every d^l_{m m'}(beta), -l <= m' <= l,
at one l) and of the spherical harmonics (d^l_{m0} with the Y_l^m normalisation), through
the C-ABI.  The kernel runs Eq. mrec in m' from both edges; the oracle ends one l-chain per
element, so the two routes share nothing.  Bar: 1e-11 absolute, widened to the l-chain
rounding bound ~ l eps / sin beta at angles close to the poles."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
BETAS = np.array([0.0, math.pi, 1e-3, math.pi - 1e-3, 0.05, 0.3, 1.2, math.pi / 2, 2.0, 2.9])


def tol(l, beta):
    s = math.sin(beta)
    bound = 8.0 * (l + 1) * min(l + 1, 1.0 / s if s > 0 else l + 1) * EPS
    return max(1e-11, 2.0 * bound)


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import wigner
    wigner.load()
    return wigner


@pytest.mark.parametrize("l,m_max", [(0, 0), (1, 1), (2, 2), (17, 17), (150, 150), (300, 40), (333, 0)])
def test_matrix_matches_oracle(W, l, m_max):
    d = W.wigner_d_matrix(torch.from_numpy(BETAS).cuda(), l, m_max).cpu().numpy()  # [j][m][m'+l]
    W.check_device_status()
    ref = O.d_matrix(l, m_max, BETAS)  # [m][m'+l][j]
    for j, b in enumerate(BETAS):
        err = np.max(np.abs(d[j] - ref[:, :, j]))
        assert err <= tol(l, b), (b, err)


def test_matrix_l4096_rows_orthonormal_and_sampled(W):
    l, m_max = 4096, 24
    beta = np.array([0.02, 0.7, 1.9, 3.1])
    d = W.wigner_d_matrix(torch.from_numpy(beta).cuda(), l, m_max)
    W.check_device_status()
    for j, b in enumerate(beta):
        h = d[j]
        gram = (h @ h.T).cpu().numpy()
        assert np.max(np.abs(gram - np.eye(m_max + 1))) <= 1e-11, b
    rng = np.random.default_rng(3)
    dh = d.cpu().numpy()
    for _ in range(40):
        m, mp, j = int(rng.integers(0, m_max + 1)), int(rng.integers(-l, l + 1)), int(rng.integers(0, 4))
        want = O.d_single(l, m, mp, float(beta[j]))
        assert abs(dh[j, m, mp + l] - want) <= tol(l, beta[j]), (m, mp, beta[j])


def test_matrix_counters_and_empty(W):
    l, m_max, nb = 64, 10, 37
    beta = torch.linspace(0.01, 3.1, nb, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    W.wigner_d_matrix(beta, l, m_max, counters=cnt)
    assert int(cnt[0]) == (m_max + 1) * (2 * l + 1) * nb
    assert W.wigner_d_matrix(beta[:0], l, m_max).shape == (0, m_max + 1, 2 * l + 1)


def test_matrix_one_angle_many_rows(W):
    """The use the evaluator is for: every row of one matrix at a large l, one angle."""
    l = 2000
    b = np.array([0.37])
    d = W.wigner_d_matrix(torch.from_numpy(b).cuda(), l).cpu().numpy()[0]
    W.check_device_status()
    assert np.max(np.abs(d @ d.T - np.eye(l + 1))) <= 1e-10
    rng = np.random.default_rng(8)
    for _ in range(30):
        m, mp = int(rng.integers(0, l + 1)), int(rng.integers(-l, l + 1))
        assert abs(d[m, mp + l] - O.d_single(l, m, mp, 0.37)) <= tol(l, 0.37), (m, mp)


def test_matrix_bad_angle_is_nan(W):
    beta = torch.tensor([0.5, -0.1, 4.0], dtype=torch.float64, device="cuda")
    d = W.wigner_d_matrix(beta, 10, 3).cpu().numpy()
    with pytest.raises(W.WignerError):
        W.check_device_status()
    assert np.all(np.isnan(d[1:])) and np.all(np.isfinite(d[0]))


@pytest.mark.parametrize("l_max,m_max", [(0, 0), (40, 12), (700, 30)])
def test_ylm_matches_oracle(W, l_max, m_max):
    theta = np.array([0.0, 0.02, 0.9, 1.7, 3.0, math.pi])
    y = W.wigner_ylm(torch.from_numpy(theta).cuda(), l_max, m_max).cpu().numpy()
    W.check_device_status()
    norm = np.sqrt((2 * np.arange(l_max + 1) + 1) / (4 * math.pi))
    ref = O.d_table(l_max, m_max, 0, theta)[:, 0] * norm[None, :, None]
    for j, b in enumerate(theta):
        assert np.max(np.abs(y[:, :, j] - ref[:, :, j])) <= max(1e-11, norm[-1] * tol(l_max, b)), b
