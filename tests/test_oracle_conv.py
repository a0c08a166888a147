"""Pins of the oracle's weighted l-sum (Eq. convdef) and of its gradients.

* Gauss-Legendre projection recovers the weights: sum_j W_j d^{l'}(b_j) C(b_j)
  = 2/(2l'+1) conj(b_{l'}) a_{l'} when every l + l' < 2N (orthogonality of the d^l).
* At beta = 0, d = delta (Sec. 4.2.1): C_{m m'} = delta_{m m'} sum_l conj(b_lm) a_lm.
* At beta = pi, d_{m m'} = (-1)^{l-m'} delta_{m,-m'}: only C_00 = sum (-1)^l conj(b) a survives.
* Linearity in a, conjugate-linearity in b.
* Gradients of L = sum |C - T|^2: central differences in a and b are exact up to
  rounding (L is quadratic in each), and in beta agree to O(h^2); the tangent-linear
  beta-derivative also matches Eq. mrec's derivative relation evaluated on the d-table.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1002_1050_gb300.inputs import beam_blm, beta_gauss_legendre, beta_uniform, sky_alm


def _inputs(L, MB, MS, seed=0):
    rng = np.random.default_rng(seed + 100)
    a = sky_alm(L, MS, seed)
    b = beam_blm(L, MB, fwhm=0.05) + 0.1j * rng.standard_normal((L + 1, MB + 1))  # complex beam too
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    return a, b


def test_gl_projection_recovers_weights():
    N = 48
    beta, W = beta_gauss_legendre(N)
    L, MB, MS = N - 1, 3, 12
    a, b = _inputs(L, MB, MS)
    C = O.conv_sum(L, MB, MS, beta, a, b)
    d = O.d_table(L, MB, MS, beta)
    for mb in range(MB + 1):
        for ms in range(MS + 1):
            proj = d[mb, ms] @ (W * C[mb, ms])  # [L+1]
            l0 = max(mb, ms)
            want = np.array([2.0 / (2 * l + 1) * np.conj(b[l, mb]) * a[l, ms] if l >= l0 else 0.0
                             for l in range(L + 1)])
            np.testing.assert_allclose(proj, want, rtol=0, atol=1e-14)


def test_beta_zero_and_pi_closed_forms():
    L, MB, MS = 80, 4, 30
    a, b = _inputs(L, MB, MS, seed=3)
    C = O.conv_sum(L, MB, MS, np.array([0.0, math.pi]), a, b)
    for mb in range(MB + 1):
        for ms in range(MS + 1):
            want0 = np.sum(np.conj(b[mb:, mb]) * a[mb:, ms]) if mb == ms else 0.0
            assert abs(C[mb, ms, 0] - want0) < 1e-13
            if mb == 0 and ms == 0:
                sgn = (-1.0) ** np.arange(L + 1)
                wantpi = np.sum(sgn * np.conj(b[:, 0]) * a[:, 0])
            else:
                wantpi = 0.0
            assert abs(C[mb, ms, 1] - wantpi) < 1e-13


def test_linearity():
    L, MB, MS = 60, 2, 40
    beta = beta_uniform(17, 0.01, math.pi - 0.01, 5)
    a1, b1 = _inputs(L, MB, MS, 1)
    a2, b2 = _inputs(L, MB, MS, 2)
    C = O.conv_sum(L, MB, MS, beta, a1 + 2.5j * a2, b1)
    np.testing.assert_allclose(C, O.conv_sum(L, MB, MS, beta, a1, b1) + 2.5j * O.conv_sum(L, MB, MS, beta, a2, b1),
                               rtol=0, atol=1e-13)
    C = O.conv_sum(L, MB, MS, beta, a1, b1 + 1.5j * b2)
    np.testing.assert_allclose(C, O.conv_sum(L, MB, MS, beta, a1, b1) - 1.5j * O.conv_sum(L, MB, MS, beta, a1, b2),
                               rtol=0, atol=1e-13)


def test_sampled_equals_full():
    L, MB, MS = 70, 3, 50
    beta = beta_uniform(9, 0.01, math.pi - 0.01, 7)
    a, b = _inputs(L, MB, MS, 4)
    C = O.conv_sum(L, MB, MS, beta, a, b)
    idx = np.array([[0, 0, 0], [3, 50, 8], [2, 17, 4], [1, 1, 1]])
    got = O.conv_sum_sampled(L, MB, MS, beta, a, b, idx)
    want = np.array([C[i, j, k] for i, j, k in idx])
    assert np.array_equal(got, want)


def _loss(L, MB, MS, beta, a, b, T):
    C = O.conv_sum(L, MB, MS, beta, a, b)
    return float(np.sum(np.abs(C - T) ** 2)), C


@pytest.fixture(scope="module")
def grad_case():
    L, MB, MS, NB = 24, 3, 24, 7
    beta = beta_uniform(NB, 0.01, math.pi - 0.01, 0)
    a, b = _inputs(L, MB, MS, 0)
    a2, _ = _inputs(L, MB, MS, 1)
    T = O.conv_sum(L, MB, MS, beta, a2, b)
    loss, C = _loss(L, MB, MS, beta, a, b, T)
    G = 2.0 * (C - T)
    ga, gb, gbeta = O.conv_grad(L, MB, MS, beta, a, b, G)
    return dict(L=L, MB=MB, MS=MS, beta=beta, a=a, b=b, T=T, ga=ga, gb=gb, gbeta=gbeta)


def test_grad_a_b_central_differences(grad_case):
    c = grad_case
    L, MB, MS, beta, T = c["L"], c["MB"], c["MS"], c["beta"], c["T"]
    h = 1e-3  # L is quadratic in a and in b: central differences carry no truncation error
    rng = np.random.default_rng(9)
    for _ in range(12):
        l = int(rng.integers(0, L + 1))
        ms = int(rng.integers(0, min(l, MS) + 1))
        for unit in (1.0, 1j):
            ap, am = c["a"].copy(), c["a"].copy()
            ap[l, ms] += h * unit
            am[l, ms] -= h * unit
            fd = (_loss(L, MB, MS, beta, ap, c["b"], T)[0] - _loss(L, MB, MS, beta, am, c["b"], T)[0]) / (2 * h)
            g = c["ga"][l, ms].real if unit == 1.0 else c["ga"][l, ms].imag
            assert abs(fd - g) <= 1e-9 * max(1.0, np.max(np.abs(c["ga"])))
        mb = int(rng.integers(0, min(l, MB) + 1))
        for unit in (1.0, 1j):
            bp, bm = c["b"].copy(), c["b"].copy()
            bp[l, mb] += h * unit
            bm[l, mb] -= h * unit
            fd = (_loss(L, MB, MS, beta, c["a"], bp, T)[0] - _loss(L, MB, MS, beta, c["a"], bm, T)[0]) / (2 * h)
            g = c["gb"][l, mb].real if unit == 1.0 else c["gb"][l, mb].imag
            assert abs(fd - g) <= 1e-9 * max(1.0, np.max(np.abs(c["gb"])))


def test_grad_beta_central_differences(grad_case):
    c = grad_case
    L, MB, MS, T = c["L"], c["MB"], c["MS"], c["T"]
    h = 1e-6
    for j in range(c["beta"].size):
        bp, bm = c["beta"].copy(), c["beta"].copy()
        bp[j] += h
        bm[j] -= h
        fd = (_loss(L, MB, MS, bp, c["a"], c["b"], T)[0] - _loss(L, MB, MS, bm, c["a"], c["b"], T)[0]) / (2 * h)
        assert abs(fd - c["gbeta"][j]) <= 1e-6 * max(1.0, abs(c["gbeta"][j]))


def test_tangent_linear_matches_mrec_derivative():
    """d/dbeta d^l_{m m'} = ((m' cos b - m)/sin b) d_{m m'} - sqrt((l-m')(l+m'+1)) d_{m,m'+1}.

    Checked through the gradient: with G = 1 at one (m_b, m_sky, beta) and zero elsewhere,
    grad_beta = Re sum_l w_l d/dbeta d^l, compared with the same sum built from Eq. mrec's
    relation on the oracle's d-table.
    """
    L, MB, MS = 40, 2, 10
    beta = np.array([0.6, 1.7, 2.5])
    a, b = _inputs(L, MB, MS + 1, 5)
    d = O.d_table(L, MB, MS + 1, beta)
    for mb in range(MB + 1):
        for ms in range(MS + 1):
            G = np.zeros((MB + 1, MS + 1, beta.size), dtype=np.complex128)
            G[mb, ms, :] = 1.0
            _, _, gbeta = O.conv_grad(L, MB, MS, beta, a[:, :MS + 1], b, G, want_a=False, want_b=False)
            l = np.arange(L + 1)[:, None]
            coef = np.sqrt(np.maximum((l - ms) * (l + ms + 1), 0))
            dd = (ms * np.cos(beta) - mb) / np.sin(beta) * d[mb, ms] - coef * d[mb, ms + 1]
            w = np.conj(b[:, mb]) * a[:, ms]
            want = np.real(np.sum(w[:, None] * dd, axis=0))
            np.testing.assert_allclose(gbeta, want, rtol=1e-10, atol=1e-12)
