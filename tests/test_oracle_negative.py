"""Pins of the oracle's negative orders, used by the full sum over every sky order
(the conviqt data cube of Sec. 4.1, Eq. conviqt, m_sky from -l_max to l_max).

The oracle runs a chain of its own for a negative order, from the general edge seed
of Sec. 3.2 (Eqs. ini1-ini2: the edges m' = -l and m = -l as well).  These tests tie it
to the explicit factorial sum at every order of l <= 12, to long chains of mpmath's
Jacobi form, to a brute-force sum of exact d values, and check that its positive half
equals the existing sum and that the corrected pi - beta identity (appendix) links the
two routes.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I
from wigner_exact import d_jacobi_mp, d_mp

EPS = np.finfo(np.float64).eps
BETAS = [1e-3, 0.3, 2.0 * math.atan2(4, 3), 1.2, math.pi / 2, 2.2, math.pi - 1e-3]


def test_small_l_negative_orders_vs_factorial_sum():
    """Every l <= 12 and every order pair with m < 0 or m' < 0 (|m|, |m'| <= l)."""
    for b in BETAS:
        tol = 2e-15 if 0.25 < b < math.pi - 0.25 else 1e-14
        worst = 0.0
        for l in range(13):
            for m in range(-l, l + 1):
                for mp in range(-l, l + 1):
                    if m >= 0 and mp >= 0:
                        continue
                    want = float(d_mp(l, m, mp, b, 40))
                    worst = max(worst, abs(O.d_single(l, m, mp, b) - want))
        assert worst <= tol, (b, worst)


@pytest.mark.parametrize("l,m,mp,beta", [
    (4096, 8, -3000, 0.9), (2048, 0, -2048, 1.6), (3000, 16, -16, 2.4), (1000, 9, -1, 0.05),
    (6000, 4, -5000, 1.4), (2500, 12, -700, 2.9),
])
def test_long_negative_chains_vs_jacobi_mp(l, m, mp, beta):
    want = d_jacobi_mp(l, m, mp, beta, 40)
    got = O.d_single(l, m, mp, beta)
    bound = 8.0 * (l + 1) * min(l + 1, 1.0 / math.sin(beta)) * EPS
    assert abs(float(want) - got) <= max(bound * max(1.0, abs(float(want))), 1e-15)


def test_full_sum_positive_half_is_the_sum():
    L, MB, MS = 60, 3, 40
    beta = I.beta_gauss_legendre(33)[0]
    a, b = I.sky_alm(L, MS, 3), I.beam_blm(L, MB, fwhm=0.1)
    full = O.conv_sum_full(L, MB, MS, beta, a, b)
    assert np.array_equal(full[:, MS:, :], O.conv_sum(L, MB, MS, beta, a, b))


def test_full_sum_negative_orders_brute_force():
    """C_{m_b,-m} = sum_l conj(b_{l m_b}) (-1)^m conj(a_{l m}) d^l_{m_b,-m}, d from the factorial sum."""
    L, MB, MS = 9, 2, 7
    beta = np.array([0.4, 1.3, 2.7])
    rng = np.random.default_rng(5)
    a = rng.standard_normal((L + 1, MS + 1)) + 1j * rng.standard_normal((L + 1, MS + 1))
    b = rng.standard_normal((L + 1, MB + 1)) + 1j * rng.standard_normal((L + 1, MB + 1))
    full = O.conv_sum_full(L, MB, MS, beta, a, b)
    for mb in range(MB + 1):
        for m in range(1, MS + 1):
            for j, bt in enumerate(beta):
                want = sum(np.conj(b[l, mb]) * (-1) ** m * np.conj(a[l, m]) * float(d_mp(l, mb, -m, bt, 40))
                           for l in range(max(mb, m), L + 1))
                assert abs(full[mb, MS - m, j] - want) <= 1e-13 * max(1.0, abs(want))


def test_full_sum_pi_minus_beta_identity():
    """C_{m_b,-m}(pi - beta) = sum_l conj(b) (-1)^m conj(a_{l m}) (-1)^{l+m_b} d^l_{m_b m}(beta):
    the negative orders' own chains against the positive chains through the corrected identity."""
    L, MB, MS = 80, 4, 60
    beta = I.beta_uniform(17, 0.05, math.pi - 0.05, 6)
    a, b = I.sky_alm(L, MS, 7), I.beam_blm(L, MB, fwhm=0.1) + 0.1j
    full = O.conv_sum_full(L, MB, MS, math.pi - beta, a, b)
    d = O.d_table(L, MB, MS, beta)  # [mb][ms][l][j]
    l = np.arange(L + 1)
    for mb in range(MB + 1):
        for m in range(MS + 1):
            w = np.conj(b[:, mb]) * (-1) ** m * np.conj(a[:, m]) * (-1.0) ** (l + mb)
            want = np.einsum("l,lj->j", w, d[mb, m])
            np.testing.assert_allclose(full[mb, MS - m], want, rtol=0, atol=1e-12)
