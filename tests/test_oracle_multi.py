"""Pins of the oracle's several-column sum (Eq. convdef for the polarised pairs of the
footnote of Sec. 4.1 and for Monte-Carlo skies that share a beam).

Each column is Eq. convdef on its own weights; the tests tie the oracle to a brute-force
sum over exact d values (the factorial sum), to linearity of the sum in the sky
coefficients, and to the scalar sum when only one column is present."""
import math

import numpy as np

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I
from wigner_exact import d_mp


def test_multi_columns_brute_force():
    """Three polarised pairs (T, G, C), one beam per column, against exact d values."""
    L, MB, MS = 8, 2, 6
    beta = np.array([0.3, 1.1, 2.9])
    rng = np.random.default_rng(11)
    a = rng.standard_normal((3, L + 1, MS + 1)) + 1j * rng.standard_normal((3, L + 1, MS + 1))
    b = rng.standard_normal((3, L + 1, MB + 1)) + 1j * rng.standard_normal((3, L + 1, MB + 1))
    got = O.conv_sum_multi(L, MB, MS, beta, a, b)
    tot = O.conv_sum_multi(L, MB, MS, beta, a, b, sum_cols=True)
    for mb in range(MB + 1):
        for ms in range(MS + 1):
            for j, bt in enumerate(beta):
                want = [sum(np.conj(b[k, l, mb]) * a[k, l, ms] * float(d_mp(l, mb, ms, bt, 40))
                            for l in range(max(mb, ms), L + 1)) for k in range(3)]
                for k in range(3):
                    assert abs(got[k, mb, ms, j] - want[k]) <= 1e-13 * max(1.0, abs(want[k]))
                assert abs(tot[mb, ms, j] - sum(want)) <= 1e-13 * max(1.0, abs(sum(want)))


def test_multi_shared_beam_is_linear_in_the_sky():
    """With one beam, the sum of the columns is the sum for the summed sky."""
    L, MB, MS = 200, 4, 120
    beta = I.beta_gauss_legendre(40)[0]
    a = np.stack([I.sky_alm(L, MS, s) for s in (1, 2, 3, 4, 5)])
    b = I.beam_blm(L, MB, fwhm=0.02)
    tot = O.conv_sum_multi(L, MB, MS, beta, a, b, sum_cols=True)
    ref = O.conv_sum(L, MB, MS, beta, a.sum(0), b)
    assert np.max(np.abs(tot - ref)) <= 1e-12 * max(1.0, float(np.max(np.abs(ref))))
    # scaling one column scales its output and nothing else
    a2 = a.copy()
    a2[2] *= -3.0
    c1, c2 = O.conv_sum_multi(L, MB, MS, beta, a, b), O.conv_sum_multi(L, MB, MS, beta, a2, b)
    assert np.array_equal(c2[[0, 1, 3, 4]], c1[[0, 1, 3, 4]])
    assert np.max(np.abs(c2[2] + 3.0 * c1[2])) <= 1e-12 * max(1.0, float(np.max(np.abs(c1[2]))))


def test_multi_single_column_is_the_sum():
    L, MB, MS = 50, 3, 50
    beta = I.beta_uniform(9, 0.01, math.pi - 0.01, 4)
    a, b = I.sky_alm(L, MS, 8), I.beam_blm(L, MB, fwhm=0.1)
    got = O.conv_sum_multi(L, MB, MS, beta, a[None], b)
    assert np.array_equal(got[0], O.conv_sum(L, MB, MS, beta, a, b))
