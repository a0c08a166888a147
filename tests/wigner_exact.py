"""Independent evaluators of d^l_{m m'}(beta) used to pin the oracle.

Wigner's explicit factorial sum (the closed form of the matrix element of
Eq. reducedwignerdef, in the convention fixed by the seed Eq. ini1 and by
d^l_{01} = -d^l_{10}, Sec. 3.1):

    d^l_{m m'}(beta) = sqrt((l+m)!(l-m)!(l+m')!(l-m')!)
        * sum_k (-1)^(m-m'+k) c^(2l+m'-m-2k) s^(m-m'+2k) / ((l+m'-k)! k! (m-m'+k)! (l-m-k)!)

with c = cos(beta/2), s = sin(beta/2), over every k for which all factorial
arguments are non-negative.  Two evaluations are provided:

* `d_rational(l, m, mp, c, s)` with rational c, s (c^2 + s^2 = 1, e.g. the
  Pythagorean pair 3/5, 4/5): returns (R, N) with d = R * sqrt(N) exactly
  (R a Fraction, N a non-negative integer), so identities can be checked with
  no rounding at all;
* `d_mp(l, m, mp, beta, dps)` in mpmath at `dps` digits, with beta taken as
  the exact binary value of the double (so it is the true value at that double).

Also a Jacobi-polynomial evaluation in mpmath for long chains, where the
factorial sum would cancel catastrophically.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial, isqrt

import mpmath


def _k_range(l, m, mp):
    lo = max(0, mp - m)
    hi = min(l + mp, l - m)
    return range(lo, hi + 1)


def d_rational(l: int, m: int, mp: int, c: Fraction, s: Fraction) -> tuple[Fraction, int]:
    """Exact d^l_{m m'} at rational half-angle cosine/sine: returns (R, N), d = R sqrt(N)."""
    if abs(m) > l or abs(mp) > l:
        return Fraction(0), 0
    n = factorial(l + m) * factorial(l - m) * factorial(l + mp) * factorial(l - mp)
    r = Fraction(0)
    for k in _k_range(l, m, mp):
        den = factorial(l + mp - k) * factorial(k) * factorial(m - mp + k) * factorial(l - m - k)
        sign = -1 if (m - mp + k) % 2 else 1
        r += Fraction(sign, den) * c ** (2 * l + mp - m - 2 * k) * s ** (m - mp + 2 * k)
    # pull the square part out of N so that equal values give equal (R, N)
    sq = isqrt(n)
    if sq * sq == n:
        return r * sq, 1
    return r, n


def rational_square(rn: tuple[Fraction, int]) -> Fraction:
    """d^2 for d = R sqrt(N)."""
    r, n = rn
    return r * r * n


def rational_value_mp(rn: tuple[Fraction, int], dps: int = 50):
    r, n = rn
    with mpmath.workdps(dps):
        return mpmath.mpf(r.numerator) / r.denominator * mpmath.sqrt(n)


def d_mp(l: int, m: int, mp: int, beta: float, dps: int = 50):
    """d^l_{m m'}(beta) by the factorial sum in mpmath (beta = the exact double)."""
    if abs(m) > l or abs(mp) > l:
        return mpmath.mpf(0)
    with mpmath.workdps(dps):
        b = mpmath.mpf(beta)
        c = mpmath.cos(b / 2)
        s = mpmath.sin(b / 2)
        pref = mpmath.sqrt(mpmath.factorial(l + m) * mpmath.factorial(l - m)
                           * mpmath.factorial(l + mp) * mpmath.factorial(l - mp))
        tot = mpmath.mpf(0)
        for k in _k_range(l, m, mp):
            den = (mpmath.factorial(l + mp - k) * mpmath.factorial(k)
                   * mpmath.factorial(m - mp + k) * mpmath.factorial(l - m - k))
            sign = -1 if (m - mp + k) % 2 else 1
            tot += sign * c ** (2 * l + mp - m - 2 * k) * s ** (m - mp + 2 * k) / den
        return +(pref * tot)


def d_jacobi_mp(l: int, m: int, mp: int, beta: float, dps: int = 40):
    """d^l_{m m'}(beta) through the Jacobi polynomial form, in mpmath.

    d = xi sqrt(k!(k+a+b)!/((k+a)!(k+b)!)) s^a c^b P_k^{(a,b)}(cos beta),
    k = l - max(|m|,|m'|), a = |m-m'|, b = |m+m'|, xi = 1 if m' >= m else (-1)^(m-m').
    mpmath's hypergeometric Jacobi evaluation is exact to the working precision, so
    this form serves long chains (l in the thousands).
    """
    k = l - max(abs(m), abs(mp))
    a = abs(m - mp)
    bb = abs(m + mp)
    xi = 1 if mp >= m else (-1 if (m - mp) % 2 else 1)
    with mpmath.workdps(dps + 20):
        b = mpmath.mpf(beta)
        c = mpmath.cos(b / 2)
        s = mpmath.sin(b / 2)
        norm = mpmath.sqrt(mpmath.factorial(k) * mpmath.factorial(k + a + bb)
                           / (mpmath.factorial(k + a) * mpmath.factorial(k + bb)))
        val = xi * norm * s ** a * c ** bb * mpmath.jacobi(k, a, bb, mpmath.cos(b))
    with mpmath.workdps(dps):
        return +val


def pythagorean_half_angles():
    """Rational (cos(beta/2), sin(beta/2)) pairs from Pythagorean triples."""
    return [(Fraction(3, 5), Fraction(4, 5)), (Fraction(5, 13), Fraction(12, 13)),
            (Fraction(8, 17), Fraction(15, 17)), (Fraction(20, 29), Fraction(21, 29)),
            (Fraction(4, 5), Fraction(3, 5)), (Fraction(12, 13), Fraction(5, 13))]
