"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the Wigner-d method itself: it only draws the
angle grids, the sky harmonic coefficients a_lm and the beam coefficients b_lm that
the beam convolution of Sec. 4 (Eqs. conviqt/convdef) consumes.  The paper's own
inputs (Planck LFI GRASP beams, CMB skies, Sec. 4.4) are not available, so the
stand-ins below follow the shapes and value distributions of those workloads:

* sky: a_lm complex Gaussian with power spectrum C_l = 1/(l+10)^2, a_l0 real;
* beam: flat-sky Fourier series of an elliptical Gaussian beam (FWHM 0.01 rad,
  ellipticity 0.2), real and zero for odd m;
* angles: equispaced interior grid, Gauss-Legendre nodes (scipy), or uniform draws.

Layouts are the C-ABI's: a[l][m_sky], b[l][m_b] complex128, beta[j] float64.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "beta_equispaced",
    "beta_gauss_legendre",
    "beta_uniform",
    "sky_alm",
    "beam_blm",
    "CONFIGS",
    "make_config",
    "mc_skies",
    "polarised_columns",
    "n_elements",
]


def beta_equispaced(n_beta: int) -> np.ndarray:
    """beta_j = (j+1) pi / (n_beta+1), j = 0..n_beta-1: equispaced in (0, pi), endpoints excluded."""
    j = np.arange(n_beta, dtype=np.float64)
    return (j + 1.0) * math.pi / (n_beta + 1.0)


def beta_gauss_legendre(n_beta: int) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre nodes as angles, ascending beta = arccos(x) with x descending.

    Returns (beta, weights).  Nodes and weights come from scipy's library routine.
    """
    from scipy.special import roots_legendre

    x, w = roots_legendre(n_beta)
    order = np.argsort(-x)  # descending x  ->  ascending beta
    x = x[order]
    w = w[order]
    return np.arccos(x).astype(np.float64), w.astype(np.float64)


def beta_uniform(n_beta: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n_beta angles drawn uniformly in (lo, hi) with numpy's default_rng(seed), sorted ascending."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.uniform(lo, hi, size=n_beta)).astype(np.float64)


def sky_alm(l_max: int, ms_max: int, seed: int) -> np.ndarray:
    """Sky coefficients a[l][m], 0 <= m <= ms_max, complex128, shape (l_max+1, ms_max+1).

    C_l = 1/(l+10)^2; a_l0 = sqrt(C_l) N(0,1) (real); a_lm = sqrt(C_l/2)(N + iN) for
    0 < m <= l; zero for m > l.  Draw order: a [l_max+1, ms_max+1] block of real
    parts, then a block of imaginary parts, from default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((l_max + 1, ms_max + 1))
    im = rng.standard_normal((l_max + 1, ms_max + 1))
    l = np.arange(l_max + 1, dtype=np.float64)[:, None]
    m = np.arange(ms_max + 1)[None, :]
    cl = 1.0 / (l + 10.0) ** 2
    a = np.sqrt(cl / 2.0) * (re + 1j * im)
    a[:, 0] = np.sqrt(cl[:, 0]) * re[:, 0]
    a[np.broadcast_to(m > np.arange(l_max + 1)[:, None], a.shape)] = 0.0
    return np.ascontiguousarray(a.astype(np.complex128))


def beam_blm(l_max: int, mb_max: int, fwhm: float = 0.01, ellipticity: float = 0.2) -> np.ndarray:
    """Beam coefficients b[l][m], 0 <= m <= mb_max, complex128 (real values), shape (l_max+1, mb_max+1).

    Elliptical Gaussian with mean width sigma = fwhm / sqrt(8 ln 2) and axis ratio
    sigma_y/sigma_x = 1 - e.  In the flat-sky limit its harmonic coefficients are
    b_lm = sqrt((2l+1)/4pi) (-1)^(m/2) exp(-(A_l - z_l)) ive(m/2, z_l) for even m,
    0 for odd m, with A_l = l(l+1)(sx^2+sy^2)/4 and z_l = l(l+1)(sx^2-sy^2)/4
    (Jacobi-Anger expansion of exp(z cos 2phi), scaled Bessel ive = exp(-z) I).
    Zero for m > l.
    """
    from scipy.special import ive

    sigma = fwhm / math.sqrt(8.0 * math.log(2.0))
    sx = sigma / math.sqrt(1.0 - ellipticity)
    sy = sigma * math.sqrt(1.0 - ellipticity)
    l = np.arange(l_max + 1, dtype=np.float64)
    ll1 = l * (l + 1.0)
    a_l = ll1 * (sx * sx + sy * sy) / 4.0
    z_l = ll1 * (sx * sx - sy * sy) / 4.0
    norm = np.sqrt((2.0 * l + 1.0) / (4.0 * math.pi))
    b = np.zeros((l_max + 1, mb_max + 1), dtype=np.float64)
    for m in range(0, mb_max + 1, 2):
        sign = -1.0 if (m // 2) % 2 else 1.0
        b[:, m] = norm * sign * np.exp(-(a_l - z_l)) * ive(m // 2, z_l)
    b[np.arange(mb_max + 1)[None, :] > np.arange(l_max + 1)[:, None]] = 0.0
    return np.ascontiguousarray(b.astype(np.complex128))


# The five workloads: a d-table, the fused FP64 sum, the FP32-carry form, the
# gradient workload and a batch of uneven instances.
CONFIGS = {
    "dtable_l256": dict(l_max=256, mb_max=4, ms_max=256, n_beta=64, grid="equispaced", seed=0),
    "conv_fp64_l4096": dict(l_max=4096, mb_max=8, ms_max=4096, n_beta=2048, grid="gl", seed=0),
    "conv_fp32x_l8192": dict(l_max=8192, mb_max=16, ms_max=8192, n_beta=8192, grid="gl", seed=0),
    "grad_l2048": dict(l_max=2048, mb_max=8, ms_max=2048, n_beta=1024, grid="uniform", seed=0, target_seed=1),
}


def mc_skies(l_max: int, ms_max: int, n: int, seed: int) -> np.ndarray:
    """n independent skies (a Monte-Carlo batch sharing one beam): sky_alm with seeds
    seed, seed + 1, ...; complex128 (n, l_max+1, ms_max+1)."""
    return np.ascontiguousarray(np.stack([sky_alm(l_max, ms_max, seed + k) for k in range(n)]))


def polarised_columns(l_max: int, mb_max: int, ms_max: int, seed: int):
    """Three (sky, beam) pairs standing for (T, G, C) of a polarised convolution: skies with
    the sky_alm spectrum at relative amplitudes 1, 0.1 and 0.02, the elliptical beam for T
    and, for G and C, beams of the same profile carried mostly at beam order 2 (ellipticity
    0.3 and 0.1, C with a quarter-turn phase).  Returns a (3, l_max+1, ms_max+1) and
    b (3, l_max+1, mb_max+1), complex128."""
    a = np.stack([sky_alm(l_max, ms_max, seed + k) * amp for k, amp in enumerate((1.0, 0.1, 0.02))])
    bt = beam_blm(l_max, mb_max)
    bg = beam_blm(l_max, mb_max, ellipticity=0.3)
    bc = 1j * beam_blm(l_max, mb_max, ellipticity=0.1)
    for bb in (bg, bc):
        if mb_max >= 2:
            bb[:, 0] *= 0.05  # mostly order 2: the spin-2 part of a polarised beam
    b = np.stack([bt, bg, bc])
    return np.ascontiguousarray(a), np.ascontiguousarray(b)


def make_config(name: str, n_beta: int | None = None, beta_slice: slice | None = None):
    """Return (l_max, mb_max, ms_max, beta, a, b) for a named workload.

    n_beta overrides the angle count (same grid rule); beta_slice selects a subset
    of the grid's angles (used to shard or sample a workload).
    """
    c = dict(CONFIGS[name])
    nb = c["n_beta"] if n_beta is None else n_beta
    if c["grid"] == "equispaced":
        beta = beta_equispaced(nb)
    elif c["grid"] == "gl":
        beta = beta_gauss_legendre(nb)[0]
    else:
        beta = beta_uniform(nb, 0.01, math.pi - 0.01, c["seed"])
    if beta_slice is not None:
        beta = np.ascontiguousarray(beta[beta_slice])
    a = sky_alm(c["l_max"], c["ms_max"], c["seed"])
    b = beam_blm(c["l_max"], c["mb_max"])
    return c["l_max"], c["mb_max"], c["ms_max"], beta, a, b


def batch_instances(n: int = 64, seed: int = 0, l_range=(128, 8192), nb_range=(32, 4096),
                    m_choices=(0, 2, 4, 8, 16)):
    """Uneven batch of fused-sum problems (the batched workload).

    Instance i draws, from default_rng(seed + i): l_max ~ U[l_range] (integers),
    mb_max from m_choices (clipped to l_max), n_beta ~ U[nb_range] (integers) on
    Gauss-Legendre nodes, and the form (0 = FP64, 1 = FP32) with probability 1/2.
    ms_max = l_max.  All instances share one seeded sky (seed) truncated to their l_max,
    and the elliptical beam of the other workloads.  Returns a list of dicts with keys
    l_max, mb_max, ms_max, n_beta, form, beta (numpy), plus the shared sky `a_full`
    (complex128 [L+1][L+1] for the largest l_max) under key "a_full" of the first dict.
    """
    specs = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        l_max = int(rng.integers(l_range[0], l_range[1] + 1))
        mb = min(int(rng.choice(m_choices)), l_max)
        nb = int(rng.integers(nb_range[0], nb_range[1] + 1))
        form = int(rng.random() < 0.5)
        specs.append(dict(l_max=l_max, mb_max=mb, ms_max=l_max, n_beta=nb, form=form,
                          beta=beta_gauss_legendre(nb)[0]))
    lmax = max(sp["l_max"] for sp in specs) if specs else 0
    if specs:
        specs[0]["a_full"] = sky_alm(lmax, lmax, seed)
    return specs


def n_elements(l_max: int, mb_max: int, ms_max: int, n_beta: int) -> int:
    """Number of (beta, m_b, m_sky, l) elements with max(m_b, m_sky) <= l <= l_max."""
    total = 0
    for mb in range(mb_max + 1):
        ms = np.arange(ms_max + 1)
        l0 = np.maximum(ms, mb)
        total += int(np.sum(np.maximum(l_max + 1 - l0, 0)))
    return total * n_beta
