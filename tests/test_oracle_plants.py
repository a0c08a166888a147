"""The pins have teeth: copies of the oracle with one planted mistake each fail them.

Each plant (ORACLE_PLANT=k in oracle/wigner_oracle.c, built into a separate
library on the CPU) is a plausible slip: a dropped d^{l-1} term, a lost seed
sign, cos for sin in the seed, a coefficient one order off, a pair not
rescaled jointly, an unconjugated beam, a wrong beam column, the wrong sign of the
cos term in the l_min cut (Eq. lmin), the (-1)^m of the real-sky relation dropped in
the sum over every sky order, the orders of a full-matrix element swapped.  The battery below
re-runs a compact version of the pins; the real oracle passes every check and
every planted copy fails at least one.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1002_1050_gb300.inputs import beta_gauss_legendre, sky_alm
from wigner_exact import d_jacobi_mp, d_mp

BETAS = np.array([0.3, 1.2, 2.2, 2.9])


def _small_exact(orc):
    L = 6
    d = orc.d_table(L, L, L, BETAS)
    for j, b in enumerate(BETAS):
        for m in range(L + 1):
            for mp in range(L + 1):
                for l in range(max(m, mp), L + 1):
                    if abs(d[m, mp, l, j] - float(d_mp(l, m, mp, float(b), 30))) > 1e-13:
                        return False
    return True


def _long_scaled_chain(orc):
    for (l, m, mp, b) in [(2000, 2, 1500, 0.6), (3000, 3, 1500, 2.6)]:
        want = float(d_jacobi_mp(l, m, mp, b, 30))
        got = orc.d_single(l, m, mp, b)
        if abs(want - got) > 1e-10 * max(1.0, abs(want)):
            return False
    return True


def _complex_beam():
    L, MB, MS = 30, 3, 10
    rng = np.random.default_rng(1)
    a = sky_alm(L, MS, 2)
    b = rng.standard_normal((L + 1, MB + 1)) + 1j * rng.standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    return L, MB, MS, a, b


def _conv_beta_zero(orc):
    L, MB, MS, a, b = _complex_beam()
    C = orc.conv_sum(L, MB, MS, np.array([0.0]), a, b)
    for mb in range(MB + 1):
        for ms in range(MS + 1):
            want = np.sum(np.conj(b[mb:, mb]) * a[mb:, ms]) if mb == ms else 0.0
            if abs(C[mb, ms, 0] - want) > 1e-12:
                return False
    return True


def _conv_gl_projection(orc):
    L, MB, MS, a, b = _complex_beam()
    beta, W = beta_gauss_legendre(L + 1)
    C = orc.conv_sum(L, MB, MS, beta, a, b)
    d = O.d_table(L, MB, MS, beta)  # the real oracle's d-table, pinned separately
    for mb in range(MB + 1):
        for ms in range(MS + 1):
            proj = d[mb, ms] @ (W * C[mb, ms])
            want = np.array([2.0 / (2 * l + 1) * np.conj(b[l, mb]) * a[l, ms] if l >= max(mb, ms) else 0.0
                             for l in range(L + 1)])
            if np.max(np.abs(proj - want)) > 1e-12:
                return False
    return True


def _lmin_turning_point(orc):
    """The cut at offset 0 sits at the exact turning point of Eq. lmin's first line."""
    for mb, ms, b in [(8, 1000, 1.0), (16, 1500, 0.9), (4, 700, 2.2)]:
        q = ms * ms + mb * mb - 2.0 * ms * mb * math.cos(b)
        l_tp = -0.5 + 0.5 * math.sqrt(1.0 + 4.0 * q / math.sin(b) ** 2)
        if not 0.0 <= orc.l_first(100000, mb, ms, b, 0.0) - l_tp <= 1.5:
            return False
    return True


def _full_sum_negative_orders(orc):
    """The negative sky orders against the sum written out with exact d values."""
    L, MB, MS = 6, 1, 4
    beta = np.array([0.7, 2.1])
    rng = np.random.default_rng(12)
    a = rng.standard_normal((L + 1, MS + 1)) + 1j * rng.standard_normal((L + 1, MS + 1))
    b = rng.standard_normal((L + 1, MB + 1)) + 1j * rng.standard_normal((L + 1, MB + 1))
    full = orc.conv_sum_full(L, MB, MS, beta, a, b)
    for mb in range(MB + 1):
        for m in range(1, MS + 1):
            for j, bt in enumerate(beta):
                want = sum(np.conj(b[l, mb]) * (-1) ** m * np.conj(a[l, m]) * float(d_mp(l, mb, -m, bt, 30))
                           for l in range(max(mb, m), L + 1))
                if abs(full[mb, MS - m, j] - want) > 1e-12 * max(1.0, abs(want)):
                    return False
    return True


def _matrix_l1(orc):
    """The rows of d^1 in closed form (d^1_{10} = -sin b / sqrt 2)."""
    b = 0.83
    c, s = math.cos(b), math.sin(b)
    want = np.array([[-s / math.sqrt(2), c, s / math.sqrt(2)], [(1 - c) / 2, -s / math.sqrt(2), (1 + c) / 2]])
    return np.max(np.abs(orc.d_matrix(1, 1, np.array([b]))[:, :, 0] - want)) <= 1e-15


BATTERY = [_small_exact, _long_scaled_chain, _conv_beta_zero, _conv_gl_projection, _lmin_turning_point,
           _full_sum_negative_orders, _matrix_l1]


def test_real_oracle_passes_battery():
    for chk in BATTERY:
        assert chk(O), chk.__name__


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_planted_mistake_is_caught(plant):
    orc = O.Planted(plant)
    assert not all(chk(orc) for chk in BATTERY), f"plant {plant} slipped through every pin"
