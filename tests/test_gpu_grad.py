"""GPU adjoint kernels: against the oracle's gradients (a different route for d/dbeta:
the tangent-linear recursion, vs the kernels' Eq. mrec neighbour chain), against
torch.autograd.gradcheck, and against central finite differences at the full
2048/8/2048/1024-angle gradient workload (32 entries, h = 1e-6 for beta).
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import autograd as AG
    from paper_1002_1050_gb300 import wigner as W
    W.load()
    return W, AG


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _complex_beam(L, MB, seed, fwhm=0.05):
    rng = np.random.default_rng(seed)
    b = I.beam_blm(L, MB, fwhm=fwhm) + 0.05j * rng.standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    return np.ascontiguousarray(b)


@pytest.mark.parametrize("L,MB,MS,NB", [(40, 3, 40, 37), (90, 6, 60, 300), (64, 8, 64, 513)])
def test_conv_backward_matches_oracle(mods, L, MB, MS, NB):
    W, _ = mods
    beta = I.beta_uniform(NB, 0.02, math.pi - 0.02, 4)
    a = I.sky_alm(L, MS, 7)
    b = _complex_beam(L, MB, 8)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((MB + 1, MS + 1, NB)) + 1j * rng.standard_normal((MB + 1, MS + 1, NB))
    C = O.conv_sum(L, MB, MS, beta, a, b)
    ga_o, gb_o, gbeta_o = O.conv_grad(L, MB, MS, beta, a, b, G)
    ga, gb, gbeta = W.wigner_conv_sum_backward(_cuda(beta), _cuda(a), _cuda(b), _cuda(C), _cuda(G))
    W.check_device_status()
    for got, ref in ((ga, ga_o), (gb, gb_o), (gbeta, gbeta_o)):
        got = got.cpu().numpy()
        scale = max(1.0, float(np.max(np.abs(ref))))
        assert np.max(np.abs(got - ref)) <= 1e-10 * scale


def test_conv_backward_subsets(mods):
    """Each gradient may be requested alone (the others are NULL)."""
    W, _ = mods
    L, MB, MS, NB = 30, 2, 20, 50
    beta = I.beta_uniform(NB, 0.1, 3.0, 1)
    a, b = I.sky_alm(L, MS, 1), _complex_beam(L, MB, 2)
    G = np.ones((MB + 1, MS + 1, NB), dtype=np.complex128)
    C = O.conv_sum(L, MB, MS, beta, a, b)
    ref = O.conv_grad(L, MB, MS, beta, a, b, G)
    for k, flags in enumerate([(True, False, False), (False, True, False), (False, False, True)]):
        out = W.wigner_conv_sum_backward(_cuda(beta), _cuda(a), _cuda(b), _cuda(C), _cuda(G), *flags)
        assert sum(o is not None for o in out) == 1
        got = out[k].cpu().numpy()
        assert np.max(np.abs(got - ref[k])) <= 1e-10 * max(1.0, np.max(np.abs(ref[k])))


def test_gradcheck_tiny(mods):
    _, AG = mods
    L, MB, MS, NB = 6, 2, 6, 4
    beta = _cuda(I.beta_uniform(NB, 0.3, 2.8, 5)).requires_grad_(True)
    a = _cuda(I.sky_alm(L, MS, 3) * 10).requires_grad_(True)
    b = _cuda(_complex_beam(L, MB, 4, fwhm=0.3)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a_, b_, be_: AG.conv_sum(a_, b_, be_), (a, b, beta),
                                    eps=1e-6, atol=1e-7, rtol=1e-6)


def test_dtable_backward_vs_oracle_differences(mods):
    W, AG = mods
    L, MB, MS, NB = 48, 3, 48, 45
    beta = I.beta_uniform(NB, 0.05, math.pi - 0.05, 9)
    rng = np.random.default_rng(1)
    G = rng.standard_normal((MB + 1, MS + 1, L + 1, NB))
    got = W.wigner_d_table_backward(_cuda(beta), _cuda(G), L, MB, MS).cpu().numpy()
    W.check_device_status()
    h = 1e-6
    ref = np.einsum("abcj,abcj->j", G, (O.d_table(L, MB, MS, beta + h) - O.d_table(L, MB, MS, beta - h)) / (2 * h))
    assert np.max(np.abs(got - ref)) <= 1e-6 * max(1.0, np.max(np.abs(ref)))
    # and through autograd
    be = _cuda(beta).requires_grad_(True)
    d = AG.d_table(be, L, MB, MS)
    (d * _cuda(G)).sum().backward()
    assert np.max(np.abs(be.grad.cpu().numpy() - got)) == 0.0


def test_grad_l2048_finite_differences(mods):
    """L = sum |C - T|^2 at the 2048/8/2048/1024-angle workload; 32 entries vs central differences."""
    W, AG = mods
    c = I.CONFIGS["grad_l2048"]
    L, MB, MS, NB = c["l_max"], c["mb_max"], c["ms_max"], c["n_beta"]
    beta_h = I.beta_uniform(NB, 0.01, math.pi - 0.01, c["seed"])
    a_h = I.sky_alm(L, MS, c["seed"])
    b_h = I.beam_blm(L, MB)
    at_h = I.sky_alm(L, MS, c["target_seed"])
    beta, a, b = _cuda(beta_h), _cuda(a_h), _cuda(b_h)
    T = W.wigner_conv_sum(beta, _cuda(at_h), b)

    a.requires_grad_(True)
    b.requires_grad_(True)
    beta.requires_grad_(True)
    loss = (AG.conv_sum(a, b, beta) - T).abs().pow(2).sum()
    loss.backward()
    W.check_device_status()
    ga, gb, gbeta = a.grad.detach(), b.grad.detach(), beta.grad.detach()

    def dloss(a2, b2, be2, a3, b3, be3):
        # L(+) - L(-) summed elementwise first, so the large common part cancels exactly per element
        Cp = W.wigner_conv_sum(be2, a2, b2)
        Cm = W.wigner_conv_sum(be3, a3, b3)
        return float(((Cp - T).abs().pow(2) - (Cm - T).abs().pow(2)).sum())

    rng = np.random.default_rng(2)
    h = 1e-6
    checks = []
    # angles: 10 entries with |g| >= 1e-3 max |g|
    gb_np = gbeta.cpu().numpy()
    cand = np.flatnonzero(np.abs(gb_np) >= 1e-3 * np.abs(gb_np).max())
    for j in rng.choice(cand, size=10, replace=False):
        bp, bm = beta.detach().clone(), beta.detach().clone()
        bp[j] += h
        bm[j] -= h
        fd = dloss(a.detach(), b.detach(), bp, a.detach(), b.detach(), bm) / (2 * h)
        checks.append((fd, gb_np[j]))
    # sky and beam: 11 entries each; real and imaginary parts are separate candidates
    for tens, g_t, n_ent in ((a, ga, 11), (b, gb, 11)):
        g_np = g_t.cpu().numpy()
        comp = np.stack([g_np.real, g_np.imag])  # [2, ...]
        cand = np.flatnonzero(np.abs(comp).ravel() >= 1e-3 * np.abs(comp).max())
        for flat in rng.choice(cand, size=n_ent, replace=False):
            part, *idx = np.unravel_index(flat, comp.shape)
            idx = tuple(idx)
            unit = 1.0 if part == 0 else 1j
            tp, tm = tens.detach().clone(), tens.detach().clone()
            tp[idx] += h * unit
            tm[idx] -= h * unit
            if tens is a:
                fd = dloss(tp, b.detach(), beta.detach(), tm, b.detach(), beta.detach()) / (2 * h)
            else:
                fd = dloss(a.detach(), tp, beta.detach(), a.detach(), tm, beta.detach()) / (2 * h)
            checks.append((fd, comp[(part,) + idx]))
    assert len(checks) == 32
    rel = [abs(fd - g) / max(abs(g), 1e-300) for fd, g in checks]
    assert max(rel) <= 1e-6, (max(rel), sorted(rel)[-5:])
