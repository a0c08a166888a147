"""Pins of the CPU oracle's d^l_{m_b m_sky}(beta) against facts outside the oracle.

Each test ties the oracle (oracle/wigner_oracle.c) to something it does not
compute itself: the explicit factorial sum (exact / 50-digit), mpmath's Jacobi
polynomials, scipy's Legendre and associated-Legendre routines, Eq. mrec (a
recursion the oracle never uses), unitarity, the appendix symmetries, the
endpoint values, Gauss-Legendre orthogonality, the exactness of power-of-two
scaling (Sec. 3.2) and the qualitative Fig. 1 statements of Sec. 2.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import eval_jacobi, eval_legendre, lpmv, gammaln

from oracle import oracle as O
from wigner_exact import d_jacobi_mp, d_mp

EPS = np.finfo(np.float64).eps
BETAS_SMALL = np.array([1e-3, 0.048, 0.3, 2.0 * math.atan2(4, 3), 1.2, math.pi / 2, 2.2, 3.0, math.pi - 1e-3])


def test_small_l_all_orders_vs_factorial_sum():
    """All l <= 12, 0 <= m_b, m_sky <= l: |oracle - exact| <= 2e-15 (1e-14 within 0.25 of a pole,
    where rounding of cos(beta) is amplified ~ 1/sin(beta))."""
    L = 12
    d = O.d_table(L, L, L, BETAS_SMALL)
    for j, b in enumerate(BETAS_SMALL):
        tol = 2e-15 if 0.25 < b < math.pi - 0.25 else 1e-14
        worst = 0.0
        for m in range(L + 1):
            for mp in range(L + 1):
                for l in range(L + 1):
                    want = float(d_mp(l, m, mp, float(b), 40)) if l >= max(m, mp) else 0.0
                    worst = max(worst, abs(d[m, mp, l, j] - want))
        assert worst <= tol, (b, worst)


@pytest.mark.parametrize("l,m,mp,beta", [
    (8192, 16, 3000, 0.5), (4096, 2, 40, 0.01), (2048, 8, 1, 1.3), (4096, 8, 4096, 1.0),
    (4096, 0, 2000, 0.6), (8192, 16, 8192, 1.9), (3000, 3, 1500, 2.6), (1000, 9, 0, 0.05),
    (6000, 4, 5000, 1.4), (300, 5, 120, 0.2), (8192, 0, 0, 0.25),
])
def test_long_chains_vs_jacobi_mp(l, m, mp, beta):
    """Sampled long chains: error within the FP64 conditioning bound ~ l eps / sin(beta)."""
    want = d_jacobi_mp(l, m, mp, beta, 40)
    got = O.d_single(l, m, mp, beta)
    bound = 8.0 * (l + 1) * min(l + 1, 1.0 / math.sin(beta)) * EPS + 1e-300
    err = abs(float(want) - got)
    assert err <= max(bound * max(1.0, abs(float(want))), 1e-15), (err, bound)
    if abs(float(want)) > 1e-280:
        assert np.sign(got) == np.sign(float(want))


def test_d00_is_legendre():
    """d^l_00(beta) = P_l(cos beta) (Eq. dl00), scipy's Legendre recurrence, l <= 2000."""
    betas = np.array([0.01, 0.5, 1.5, 2.5, 3.1])
    d = O.d_table(2000, 0, 0, betas)[0, 0]
    ref = eval_legendre(np.arange(2001)[:, None], np.cos(betas)[None, :])
    bound = 8 * 2001 * np.minimum(2001, 1 / np.sin(betas)) * EPS
    assert np.all(np.abs(d - ref) <= bound[None, :])


def test_dm0_is_associated_legendre():
    """d^l_{m0}(beta) = sqrt((l-m)!/(l+m)!) P_l^m(cos beta), Condon-Shortley phase (scipy lpmv)."""
    L, M = 60, 12
    betas = np.array([0.2, 0.9, 1.7, 2.8])
    d = O.d_table(L, M, 0, betas)
    for m in range(M + 1):
        for l in range(m, L + 1):
            norm = math.exp(0.5 * (gammaln(l - m + 1) - gammaln(l + m + 1)))
            ref = norm * lpmv(m, l, np.cos(betas))
            np.testing.assert_allclose(d[m, 0, l], ref, rtol=0, atol=1e-13)


def test_general_vs_scipy_jacobi():
    """General orders through the Jacobi form with scipy's eval_jacobi, l <= 120."""
    L = 120
    betas = np.array([0.35, 1.1, 2.4])
    d = O.d_table(L, 6, 40, betas)
    for m in range(7):
        for mp in range(0, 41, 3):
            for l in range(max(m, mp), L + 1, 7):
                k = l - max(m, mp)
                a, b = abs(m - mp), m + mp
                xi = 1.0 if mp >= m else (-1.0) ** (m - mp)
                lognorm = 0.5 * (gammaln(k + 1) + gammaln(k + a + b + 1) - gammaln(k + a + 1) - gammaln(k + b + 1))
                ref = xi * np.exp(lognorm) * np.sin(betas / 2) ** a * np.cos(betas / 2) ** b * eval_jacobi(k, a, b, np.cos(betas))
                np.testing.assert_allclose(d[m, mp, l], ref, rtol=1e-10, atol=1e-14)


def test_mrec_holds():
    """Eq. mrec, a recursion in m' that the oracle never evaluates, holds on its output."""
    L = 200
    betas = np.array([0.15, 0.8, 1.6, 2.9])
    d = O.d_table(L, 5, L, betas)
    cb, sb = np.cos(betas), np.sin(betas)
    worst = 0.0
    for m in range(6):
        for mp in range(1, L):
            for l in range(max(m, mp + 1), L + 1, 5):
                lhs = (-m + mp * cb) / sb * d[m, mp, l]
                rhs = 0.5 * math.sqrt((l + mp) * (l - mp + 1)) * d[m, mp - 1, l] \
                    + 0.5 * math.sqrt((l - mp) * (l + mp + 1)) * d[m, mp + 1, l]
                worst = max(worst, float(np.max(np.abs(lhs - rhs) * sb)))
    assert worst < 1e-11, worst


def test_unitarity():
    """sum_{m'=-l}^{l} (d^l_{m m'})^2 = 1, negative m' from d_{m,-m'}(b) = (-1)^{l+m} d_{m m'}(pi - b)."""
    L = 300
    betas = np.array([0.4, 1.3, 2.2])
    dp = O.d_table(L, 4, L, betas)
    dn = O.d_table(L, 4, L, math.pi - betas)  # d_{m m'}(pi - b) = +- d_{m,-m'}(b)
    for m in range(5):
        for l in range(m, L + 1, 13):
            tot = np.sum(dp[m, :l + 1, l] ** 2, axis=0) + np.sum(dn[m, 1:l + 1, l] ** 2, axis=0)
            np.testing.assert_allclose(tot, 1.0, rtol=0, atol=5e-13)


def test_pi_minus_beta_parity_sign():
    """d_{m,-m'}(b) = (-1)^{l+m} d_{m m'}(pi - b) with the sign, against the factorial sum (Sec. 8 reading of appendix line 7)."""
    b = 0.9
    dpi = O.d_table(10, 3, 10, np.array([math.pi - b]))
    for m in range(4):
        for mp in range(0, 11):
            for l in range(max(m, mp), 11):
                want = float(d_mp(l, m, -mp, b, 40))
                got = (-1) ** (l + m) * dpi[m, mp, l, 0]
                assert abs(want - got) < 1e-15


def test_transpose_symmetry_two_seed_branches():
    """d_{m m'} = (-1)^{m-m'} d_{m' m}: chains with m_b > m_sky and m_b < m_sky use different seeds."""
    L = 400
    betas = np.array([0.07, 1.0, 2.7])
    d = O.d_table(L, 30, 30, betas)
    for m in range(31):
        for mp in range(31):
            ph = (-1) ** (m - mp)
            np.testing.assert_allclose(d[m, mp], ph * d[mp, m], rtol=0, atol=2e-14)


def test_endpoints():
    """d(0) = delta_{m m'} (Sec. 4.2.1) and d(pi)_{m m'} = (-1)^{l-m'} delta_{m,-m'}."""
    L = 50
    d = O.d_table(L, 5, L, np.array([0.0, math.pi]))
    for m in range(6):
        for mp in range(L + 1):
            for l in range(max(m, mp), L + 1):
                want0 = 1.0 if m == mp else 0.0
                wantpi = (-1.0) ** l if (m == 0 and mp == 0) else 0.0
                assert abs(d[m, mp, l, 0] - want0) < 1e-13
                assert abs(d[m, mp, l, 1] - wantpi) < 1e-13


def test_gauss_legendre_orthogonality():
    """sum_j W_j d^l(b_j) d^l'(b_j) = 2/(2l+1) delta_{l l'}, exact for l + l' < 2N."""
    from paper_1002_1050_gb300.inputs import beta_gauss_legendre

    N = 64
    beta, w = beta_gauss_legendre(N)
    L = N - 1
    d = O.d_table(L, 3, 20, beta)
    for m in range(4):
        for mp in (0, 1, 7, 20):
            l0 = max(m, mp)
            G = (d[m, mp] * w[None, :]) @ d[m, mp].T
            want = np.diag([2.0 / (2 * l + 1) if l >= l0 else 0.0 for l in range(L + 1)])
            np.testing.assert_allclose(G, want, rtol=0, atol=1e-13)


def test_scaling_is_exact():
    """Scaled doubles (S = 2^90) equal the unscaled recurrence bit for bit where it stays in range."""
    L = 600
    betas = np.array([0.3, 1.0, 1.9, 2.8])
    ds = O.d_table(L, 6, 200, betas, scaling=True)
    du = O.d_table(L, 6, 200, betas, scaling=False)
    for m in range(7):
        for mp in range(0, 201):
            for j, b in enumerate(betas):
                l0 = max(m, mp)
                s = ds[m, mp, l0:, j]
                u = du[m, mp, l0:, j]
                # the unscaled run is valid only if its seed and every later value are normal doubles
                if abs(u[0]) < 1e-290 or not np.all(np.isfinite(u)):
                    continue
                nz = np.abs(u) > 1e-290
                assert np.array_equal(s[nz], u[nz])
    # and the scaled run reaches far below the double range where the plain one cannot
    tiny = O.d_single(4000, 0, 3990, 0.05)
    assert tiny == 0.0 or abs(tiny) < 1e-300
    big = O.d_single(8000, 2, 7600, 1.3)
    assert abs(big) > 1e-10  # classical region: O(1/sqrt(l)) despite a seed ~ 1e-1000


def _peaks(y):
    a = np.abs(y)
    return [i for i in range(1, len(a) - 1) if a[i] >= a[i - 1] and a[i] >= a[i + 1]]


def test_fig1_transitions_and_tallest_peak():
    """Sec. 2, Fig. 1: where each example turns classical, and that the tallest peak is the first after it."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig1_transitions.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        if c["vary"] == "l":
            lo, hi = c["l_range"]
            d = O.d_table(hi, c["m"], c["mp"], np.array([c["beta"]]))[c["m"], c["mp"], :, 0]
            xs = np.arange(hi + 1)
            sel = xs >= lo
            xs, y = xs[sel], d[sel]
            # Eq. classiccond with m = 0: l(l+1) >= m'^2 / sin^2 beta
            tp = xs[np.argmax(xs * (xs + 1) >= c["mp"] ** 2 / math.sin(c["beta"]) ** 2)]
            assert abs(tp - c["transition"]) <= 1
            pk = [p for p in _peaks(y) if xs[p] >= tp]
            assert xs[np.argmax(np.abs(y))] == xs[pk[0]]
        elif c["vary"] == "mp":
            l = c["l"]
            d = O.d_table(l, 0, l, np.array([c["beta"]]))[0, :, l, 0]
            mps = np.arange(l + 1)
            tp = np.max(mps[l * (l + 1) - mps ** 2 / math.sin(c["beta"]) ** 2 >= 0])
            assert abs(tp - c["transition"]) <= 1
            pk = [p for p in _peaks(d) if p <= tp]
            assert np.argmax(np.abs(d)) == pk[-1]  # first peak met coming in from the non-classical side
        else:
            l, mp = c["l"], c["mp"]
            bs = np.linspace(1e-3, c["beta_range"][1], 3000)
            d = O.d_table(l, 0, mp, bs)[0, mp, l]
            ok = l * (l + 1) - mp ** 2 / np.sin(bs) ** 2 >= 0
            tp = bs[np.argmax(ok)]
            assert abs(tp - c["transition"]) < 2e-3
            pk = [p for p in _peaks(d) if bs[p] >= tp]
            assert np.argmax(np.abs(d)) == pk[0]
