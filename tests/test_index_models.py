"""CPU models of the kernels' index arithmetic (no GPU): every output slot is written
exactly once and every access stays inside its buffer, for the launch shapes the
library uses.  Each model restates the index formulas of one kernel."""
import math

import numpy as np
import pytest


def fp64_angle_map(NT, CPT, chunk, tid, c):
    """conv_fp64_item / conv_multi_kernel: a warp holds 32 x CPT consecutive angles."""
    return chunk * NT * CPT + (tid >> 5) * (32 * CPT) + c * 32 + (tid & 31)


@pytest.mark.parametrize("NT,CPT", [(256, 2), (128, 4), (256, 1)])
def test_fp64_angle_map_is_a_permutation_of_each_chunk(NT, CPT):
    for chunk in range(3):
        got = sorted(fp64_angle_map(NT, CPT, chunk, t, c) for t in range(NT) for c in range(CPT))
        assert got == list(range(chunk * NT * CPT, (chunk + 1) * NT * CPT))
        for w in range(NT // 32):  # a warp's angles are consecutive
            a = sorted(fp64_angle_map(NT, CPT, chunk, t, c) for t in range(32 * w, 32 * w + 32) for c in range(CPT))
            assert a == list(range(a[0], a[0] + 32 * CPT))


@pytest.mark.parametrize("l", [0, 1, 2, 7, 64, 301])
def test_matrix_sides_cover_every_order_once(l):
    """dmatrix_kernel: side 0 writes m' = k for k = l .. m*, side 1 writes m' = -k for
    k = l .. 1 - m*, with m* = round(m cos beta); slots l + m' in [0, 2l]."""
    for m in range(l + 1):
        for beta in (0.0, 1e-9, 0.3, math.pi / 2, 2.5, math.pi - 1e-9, math.pi):
            mstar = int(np.rint(m * math.cos(beta)))
            assert -m <= mstar <= m
            slots = [l + k for k in range(mstar, l + 1)] + [l - k for k in range(1 - mstar, l + 1)]
            assert sorted(slots) == list(range(2 * l + 1)), (l, m, beta)


@pytest.mark.parametrize("l,TM", [(5, 32), (100, 32), (1000, 32)])
def test_matrix_tiles_and_stage_indices(l, TM):
    """Tile ts = l, l - TM, ...: table index ts - k in [0, TM), stage column the same; a
    lane's orders k in [stop, l]; the store's order ts - lane stays within [-l, l] when
    it is at or above the row's stop."""
    for stop in (-l, -l // 2, 0, 1, l // 2, l, l + 1):
        ts = l
        seen = []
        while ts >= stop:
            kend = max(ts - TM + 1, stop)
            for k in range(ts, kend - 1, -1):
                assert 0 <= ts - k < TM
                seen.append(k)
            for lane in range(32):
                k = ts - lane
                if k >= stop:
                    assert -l <= k <= l
            ts -= TM
        assert seen == list(range(l, stop - 1, -1)) if stop <= l else seen == []


@pytest.mark.parametrize("n_col", [1, 3, 4, 5, 8, 9, 13])
def test_multi_passes_cover_every_column_once(n_col):
    """wigner_conv_sum_multi: passes of up to four columns, columns k0 .. k0 + K - 1."""
    KMAX = 4
    cols = []
    for k0 in range(0, n_col, KMAX):
        K = min(KMAX, n_col - k0)
        cols += [k0 + q for q in range(K)]
    assert cols == list(range(n_col))


@pytest.mark.parametrize("mb_max,ms_max,n_beta", [(0, 0, 1), (8, 4096, 2048), (3, 40, 12), (16, 8192, 8192)])
def test_cube_scatter_reads_inside_c_and_writes_inside_z(mb_max, ms_max, n_beta):
    """cube_scatter_kernel: Z[j][p][k], p < n_a, k < n_h = n_g/2 + 1, read from
    C[mb][S + k or S - k][j]; the row p holds m_b = p (p <= M) or p - n_a (p >= n_a - M)."""
    def fft_size(n):
        m = max(1, n)
        while True:
            k = m
            for p in (2, 3, 5, 7):
                while k % p == 0:
                    k //= p
            if k == 1:
                return m
            m += 1
    na, ng = fft_size(2 * mb_max + 1), fft_size(2 * ms_max + 1)
    nh = ng // 2 + 1
    S, NS = ms_max, 2 * ms_max + 1
    for p in range(na):
        mb = p if p <= mb_max else p - na
        have = -mb_max <= mb <= mb_max
        for k in (0, min(S, nh - 1), nh - 1):
            if have and k <= S:
                row = (mb * NS + (S + k)) if mb >= 0 else ((-mb) * NS + (S - k))
                assert 0 <= row < (mb_max + 1) * NS
    # every m_b in [-M, M] lands on exactly one row
    rows = [p if p <= mb_max else p - na for p in range(na)]
    assert sorted(r for r in rows if -mb_max <= r <= mb_max) == list(range(-mb_max, mb_max + 1))
