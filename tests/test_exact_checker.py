"""Pins of the exact checker itself, in exact rational arithmetic (no rounding).

The factorial-sum evaluator in wigner_exact.py is the yardstick for the oracle,
so it is first tied to facts that do not depend on its own formula:
closed forms of d^1 (Sec. 8 convention: d^1_{10} = -sin(beta)/sqrt 2),
d^l_{ll} = cos^{2l}(beta/2), the seeds of Eqs. ini1-ini2, unitarity of d^l,
the appendix symmetries (first three lines) and the group law
d(beta1 + beta2) = d(beta1) d(beta2) of the rotation matrices (Eq. reducedwignerdef).
"""
from fractions import Fraction
from math import comb

import mpmath
import pytest

from wigner_exact import d_mp, d_rational, pythagorean_half_angles, rational_square, rational_value_mp

PAIRS = pythagorean_half_angles()


@pytest.mark.parametrize("c,s", PAIRS)
def test_d1_closed_forms(c, s):
    cosb = c * c - s * s
    # d^1_{11} = (1+cos b)/2, d^1_{1,-1} = (1-cos b)/2, d^1_{00} = cos b
    assert d_rational(1, 1, 1, c, s) == ((1 + cosb) / 2, 1)
    assert d_rational(1, 1, -1, c, s) == ((1 - cosb) / 2, 1)
    assert d_rational(1, 0, 0, c, s) == (cosb, 1)
    # d^1_{10} = -sin b / sqrt 2 = -sqrt2 c s ; d^1_{01} = +sqrt2 c s
    assert d_rational(1, 1, 0, c, s) == (-c * s, 2)
    assert d_rational(1, 0, 1, c, s) == (c * s, 2)


@pytest.mark.parametrize("c,s", PAIRS[:3])
@pytest.mark.parametrize("l", [0, 1, 2, 5, 9])
def test_extreme_rows_are_seeds(c, s, l):
    """Eqs. ini1-ini2 with the labels read as d_{l,m}, d_{-l,m}, d_{m,l}, d_{m,-l}."""
    for m in range(-l, l + 1):
        a2 = Fraction(comb(2 * l, l + m))  # A^2
        want = [
            (d_rational(l, l, m, c, s), c ** (l + m) * (-s) ** (l - m)),
            (d_rational(l, -l, m, c, s), c ** (l - m) * s ** (l + m)),
            (d_rational(l, m, l, c, s), c ** (l + m) * s ** (l - m)),
            (d_rational(l, m, -l, c, s), c ** (l - m) * (-s) ** (l + m)),
        ]
        for got, pw in want:
            assert rational_square(got) == a2 * pw * pw
            r, _ = got
            assert (r > 0) == (pw > 0) or pw == 0


@pytest.mark.parametrize("c,s", PAIRS[:4])
def test_dll_power(c, s):
    for l in range(0, 10):
        assert d_rational(l, l, l, c, s) == (c ** (2 * l), 1)
        assert rational_square(d_rational(l, l, -l, c, s)) == s ** (4 * l)


@pytest.mark.parametrize("c,s", PAIRS)
@pytest.mark.parametrize("l", [1, 2, 3, 6, 12])
def test_unitarity_exact(c, s, l):
    """sum_{m'} (d^l_{m m'})^2 = 1 for every m, exactly."""
    for m in range(-l, l + 1):
        tot = sum(rational_square(d_rational(l, m, mp, c, s)) for mp in range(-l, l + 1))
        assert tot == 1


@pytest.mark.parametrize("c,s", PAIRS[:4])
@pytest.mark.parametrize("l", [2, 5, 8])
def test_appendix_symmetries_exact(c, s, l):
    """d_{mm'} = (-1)^{m-m'} d_{-m,-m'} = (-1)^{m-m'} d_{m'm} = d_{-m',-m} (appendix A, lines 1-3)."""
    for m in range(-l, l + 1):
        for mp in range(-l, l + 1):
            r, n = d_rational(l, m, mp, c, s)
            ph = -1 if (m - mp) % 2 else 1
            r1, n1 = d_rational(l, -m, -mp, c, s)
            r2, n2 = d_rational(l, mp, m, c, s)
            r3, n3 = d_rational(l, -mp, -m, c, s)
            assert (r, n) == (ph * r1, n1) or (r == 0 and r1 == 0)
            assert (r, n) == (ph * r2, n2) or (r == 0 and r2 == 0)
            assert (r, n) == (r3, n3) or (r == 0 and r3 == 0)


def test_group_law_mp():
    """d^l(b1 + b2) = d^l(b1) d^l(b2) as matrices (rotations about one axis compose)."""
    b1, b2 = 0.7, 1.1
    for l in (1, 3, 6):
        for m in range(-l, l + 1):
            for mp in range(-l, l + 1):
                lhs = d_mp(l, m, mp, b1 + b2, dps=40)
                rhs = mpmath.fsum(d_mp(l, m, k, b1, 40) * d_mp(l, k, mp, b2, 40) for k in range(-l, l + 1))
                # b1 + b2 as a double differs from the exact sum by < 1 ulp: allow that
                assert abs(lhs - rhs) < 1e-14


def test_rational_matches_mp():
    c, s = PAIRS[0]
    beta = 2.0 * float(mpmath.atan2(4, 3))
    for l in (3, 7):
        for m in range(0, l + 1):
            for mp in range(-l, l + 1):
                v = rational_value_mp(d_rational(l, m, mp, c, s))
                w = d_mp(l, m, mp, beta, 50)
                assert abs(v - w) < 1e-15
