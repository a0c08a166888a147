"""Pins of the oracle's l_min cut (Sec. 4.2.1, Eq. lmin): in the chain (m_b, m', beta) the
terms with l < l_min = (sqrt(m'^2 + m_b^2 - 2 m' m_b cos beta) - offset) / sin beta lie in the
non-classical region and are left out; at beta = 0 the chain is left out unless m_b = m'.

The pins: the cut removes only values of one sign that grow monotonically with l (the
non-classical, exponentially rising side of the turning point) and the values beyond it
oscillate; the cut at offset 0 agrees with the exact turning point (the first line of
Eq. lmin) to one order; a large offset cuts nothing (bitwise the uncut sum); beta = 0
follows d(0) = delta; the mirror symmetry of the formula (m' -> -m', beta -> pi - beta);
and the error of the cut sum falls steeply as the offset grows, the shape of the paper's
accuracy table (Sec. 4.4)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I

CHAINS = [(0, 300, 0.3), (8, 1000, 1.0), (4, 700, 2.2), (2, 40, 0.01), (16, 1500, 0.9), (1, 200, 2.9)]


@pytest.mark.parametrize("mb,ms,beta", CHAINS)
def test_cut_region_is_non_classical(mb, ms, beta):
    """Below the cut the ratios d^{l+1}/d^l keep one sign (every l of one sign for
    beta < pi/2, alternating for beta > pi/2) and exceed 1 in magnitude; past the cut the
    ratio's sign changes (the chain oscillates)."""
    L = 2000
    lf = O.l_first(L, mb, ms, beta, 0.0)
    l0 = max(mb, ms)
    d = O.d_column(L, mb, ms, np.array([beta]))[:, 0]
    below = d[l0:min(lf, L + 1)]
    if below.size > 2:
        r = below[1:] / below[:-1]
        assert np.all(np.sign(r) == np.sign(r[0])), "ratio sign changes below the cut"
        assert np.all(np.abs(r) > 1.0), "not growing below the cut"
    if lf + 40 <= L:
        above = d[lf:lf + 200]
        r = above[1:] / above[:-1]
        assert np.any(np.sign(r) != np.sign(r[0]))


@pytest.mark.parametrize("mb,ms,beta", CHAINS[:5] + [(3, 3, 0.4), (0, 900, 1.2)])
def test_offset_zero_matches_the_turning_point(mb, ms, beta):
    """The approximate line of Eq. lmin at offset 0 against its exact first line
    l_tp = -1/2 + 1/2 sqrt(1 + 4 q / sin^2 beta), q = m'^2 + m_b^2 - 2 m' m_b cos beta:
    x = sqrt(q) / sin beta exceeds l_tp by 1/2 - O(1/x), and the cut is ceil(x)."""
    L = 100000
    q = ms * ms + mb * mb - 2.0 * ms * mb * math.cos(beta)
    l_tp = -0.5 + 0.5 * math.sqrt(1.0 + 4.0 * q / math.sin(beta) ** 2)
    lf = O.l_first(L, mb, ms, beta, 0.0)
    l0 = max(mb, ms)
    assert lf >= l0
    if lf > l0:
        assert 0.0 <= lf - l_tp <= 1.5
    else:
        assert l_tp < l0


def test_large_offset_cuts_nothing():
    L, MB, MS = 120, 4, 100
    beta = I.beta_uniform(25, 0.0, math.pi, 3)
    a, b = I.sky_alm(L, MS, 4), I.beam_blm(L, MB, fwhm=0.1)
    big = float(MB + MS)  # sqrt(q) <= m_b + m'
    assert np.array_equal(O.conv_sum(L, MB, MS, beta, a, b, offset=big), O.conv_sum(L, MB, MS, beta, a, b))
    assert np.array_equal(O.conv_sum_full(L, MB, MS, beta, a, b, offset=big),
                          O.conv_sum_full(L, MB, MS, beta, a, b))


def test_beta_zero_rule():
    L, MB, MS = 60, 5, 40
    beta = np.array([0.0, 0.7])
    a, b = I.sky_alm(L, MS, 5), I.beam_blm(L, MB, fwhm=0.1) + 0.3j
    exact = O.conv_sum(L, MB, MS, beta, a, b)
    for off in (0.0, 3.0, 1e6):
        cut = O.conv_sum(L, MB, MS, beta, a, b, offset=off)
        for mb in range(MB + 1):
            for ms in range(MS + 1):
                if mb == ms:
                    assert cut[mb, ms, 0] == exact[mb, ms, 0]
                else:
                    assert cut[mb, ms, 0] == 0
        assert O.l_first(L, 2, 3, 0.0, off) == L + 1 and O.l_first(L, 3, 3, 0.0, off) == 3


@pytest.mark.parametrize("mb,ms,beta,off", [(3, 500, 0.4, 0.0), (8, 2000, 1.3, 30.0), (1, 50, 2.8, 5.0),
                                            (6, 3000, 0.2, 200.0)])
def test_mirror_symmetry_of_the_cut(mb, ms, beta, off):
    """q(m_b, -m', pi - beta) = q(m_b, m', beta) and sin(pi - beta) = sin beta."""
    L = 5000
    assert O.l_first(L, mb, -ms, math.pi - beta, off) == O.l_first(L, mb, ms, beta, off)


def test_error_falls_with_the_offset():
    """The cut sum's error against the exact sum drops steeply and monotonically as the
    offset grows: at L = 600 from ~1e-1 (offset 0, the cut at the turning point) through
    ~1e-7 (15) to ~1e-14 (30) of max |C|."""
    L, MB, MS = 600, 6, 600
    beta = I.beta_gauss_legendre(60)[0]
    a, b = I.sky_alm(L, MS, 3), I.beam_blm(L, MB, fwhm=0.05)
    ref = O.conv_sum(L, MB, MS, beta, a, b)
    sc = float(np.max(np.abs(ref)))
    errs = [float(np.max(np.abs(O.conv_sum(L, MB, MS, beta, a, b, offset=o) - ref))) / sc
            for o in (0, 5, 10, 15, 30, 60)]
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:]))
    assert errs[0] > 1e-2 and errs[3] < 1e-5 and errs[4] < 1e-12
