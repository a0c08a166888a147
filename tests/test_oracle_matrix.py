"""Pins of the oracle's full-matrix rows d^l_{m m'}(beta), -l <= m' <= l (the evaluator of
Sec. 3.1 computes the whole matrix at one (l, beta)), and of the spherical harmonics
built from its m' = 0 column.

Each element of oracle.d_matrix is the end of its own l-chain; the pins are properties
of the rotation matrix that no single chain knows about: the rows are orthonormal
(the matrix is orthogonal), rotations compose, d_{m m'} = (-1)^{m-m'} d_{m' m}, the
three-term relation in m' (Eq. mrec) holds across neighbouring chains, the l = 1 closed
forms, and Y_l^m from the m' = 0 column equals scipy's spherical harmonic."""
import math

import numpy as np
import pytest

from oracle import oracle as O

EPS = np.finfo(np.float64).eps


def chain_bound(l, beta):
    """Rounding bound of an l-chain (Sec. 3.2): ~ l eps / sin beta near the poles."""
    return 8.0 * (l + 1) * min(l + 1, 1.0 / math.sin(beta)) * EPS


def full_matrix(l, beta):
    """The whole (2l+1) x (2l+1) matrix from rows m >= 0 and d_{-m,-m'} = (-1)^{m-m'} d_{m m'}."""
    h = O.d_matrix(l, l, np.array([beta]))[:, :, 0]  # [m][m' + l]
    full = np.empty((2 * l + 1, 2 * l + 1))
    full[l:, :] = h
    for m in range(1, l + 1):
        for mp in range(-l, l + 1):
            full[l - m, mp + l] = (-1.0) ** (m - mp) * h[m, -mp + l]
    return full


@pytest.mark.parametrize("l,beta", [(1, 0.7), (7, 0.2), (40, 1.3), (120, 2.8), (300, 0.05)])
def test_rows_are_orthonormal(l, beta):
    h = O.d_matrix(l, l, np.array([beta]))[:, :, 0]
    assert np.max(np.abs(h @ h.T - np.eye(l + 1))) <= 2.0 * chain_bound(l, beta)


def test_negative_rows_follow_and_rotations_compose():
    l = 25
    for b1, b2 in [(0.4, 0.9), (1.2, 1.5), (2.0, 0.3)]:
        f1, f2, f12 = full_matrix(l, b1), full_matrix(l, b2), full_matrix(l, b1 + b2)
        assert np.max(np.abs(f1 @ f2 - f12)) <= 1e-13
    # the negative rows used above agree with their own chains
    for m, mp in [(-3, 5), (-7, -2), (-25, 11)]:
        want = O.d_single(l, m, mp, 0.9)
        assert abs(full_matrix(l, 0.9)[m + l, mp + l] - want) <= 1e-14


@pytest.mark.parametrize("l,beta", [(30, 0.5), (200, 2.1)])
def test_transpose_symmetry(l, beta):
    h = O.d_matrix(l, l, np.array([beta]))[:, :, 0]
    for m in range(l + 1):
        for mp in range(l + 1):
            assert abs(h[m, mp + l] - (-1.0) ** (m - mp) * h[mp, m + l]) <= 1e-14


@pytest.mark.parametrize("l,beta", [(50, 0.4), (400, 1.9), (1000, 1.2)])
def test_m_recursion_holds(l, beta):
    """Eq. mrec across neighbouring elements of a row:
    2 (m' cos b - m)/sin b d_{m m'} = sqrt((l+m')(l-m'+1)) d_{m,m'-1} + sqrt((l-m')(l+m'+1)) d_{m,m'+1}."""
    m_max = min(l, 12)
    h = O.d_matrix(l, m_max, np.array([beta]))[:, :, 0]
    cb, sb = math.cos(beta), math.sin(beta)
    for m in range(m_max + 1):
        for mp in range(-l + 1, l):
            lhs = 2.0 * (mp * cb - m) / sb * h[m, mp + l]
            rhs = (math.sqrt((l + mp) * (l - mp + 1)) * h[m, mp - 1 + l]
                   + math.sqrt((l - mp) * (l + mp + 1)) * h[m, mp + 1 + l])
            assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(2.0 * (mp * cb - m) / sb)), (m, mp)


def test_first_ratio_and_l1_closed_forms():
    """The start of the ratio recursion, d_{m l} / d_{m,l-1} = sqrt(l/2) sin b / (l cos b - m), and d^1."""
    for l, m, b in [(10, 3, 0.6), (200, 0, 1.0), (57, 40, 2.5)]:
        h = O.d_matrix(l, m, np.array([b]))[m, :, 0]
        assert abs(h[2 * l] / h[2 * l - 1] - math.sqrt(l / 2) * math.sin(b) / (l * math.cos(b) - m)) <= 1e-12
    b = 0.83
    d1 = O.d_matrix(1, 1, np.array([b]))[:, :, 0]
    c, s = math.cos(b), math.sin(b)
    # d^1_{10} = -sin b / sqrt 2 (the convention of Eq. ini1), d^1_{11} = (1 + cos b)/2
    want = np.array([[-s / math.sqrt(2), c, s / math.sqrt(2)],
                     [(1 - c) / 2, -s / math.sqrt(2), (1 + c) / 2]])
    assert np.max(np.abs(d1 - want)) <= 1e-15


def test_ylm_from_the_m0_column_is_scipys():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    theta = np.array([0.1, 0.9, 1.7, 3.0])
    L, M = 40, 12
    d = O.d_table(L, M, 0, theta)[:, 0]  # [m][l][j] = d^l_{m 0}
    for l in range(L + 1):
        for m in range(min(l, M) + 1):
            ours = math.sqrt((2 * l + 1) / (4 * math.pi)) * d[m, l]
            ref = sp.sph_harm_y(l, m, theta, 0.0).real
            assert np.max(np.abs(ours - ref)) <= 1e-13, (l, m)
