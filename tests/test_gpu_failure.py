"""Failure paths on the GPU, made without faulting it.

* Bounded waits: with the wait limit of the TMA weight pipeline set to 0 tries (a host
  setting passed to the kernel), every CTA's first wait gives up at once.  The call must
  return, the device status must read WG_ERR_TIMEOUT, every output the CTAs abandoned
  must be NaN (no stale values), and with the default limit restored the same call must
  match the oracle again -- the context stays usable.
* Allocation failures: with failures injected on the host (the allocator is not called),
  the call that needed memory returns WG_ERR_ALLOC and a retry succeeds.  Run in a fresh
  process so the library has allocated nothing yet.
* Guard words: output buffers are views into larger buffers filled with a sentinel; the
  sentinel before and after each output must survive every kernel that writes it (the
  fused sums of each form, the sum over every sky order with its mirrored stores, the
  data cube's scatter, the d-table and the several-column sum).
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WG_ERR_ALLOC, WG_ERR_TIMEOUT = -3, -4


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import wigner
    wigner.load()
    return wigner


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def small():
    L, MB, MS, NB = 300, 4, 300, 700  # several tiles and chunks, ragged tails
    g = I.beta_gauss_legendre(NB)[0]
    beta = g.copy()
    beta[NB - NB // 2:] = math.pi - g[:NB // 2][::-1]  # exactly mirror-symmetric (the full sum requires it)
    a = I.sky_alm(L, MS, 2)
    b = I.beam_blm(L, MB, fwhm=0.05)
    return L, MB, MS, beta, a, b


@pytest.mark.parametrize("kind", ["fp64", "fp64s", "full", "lmin"])
def test_wait_gives_up_and_context_survives(W, small, kind):
    L, MB, MS, beta, a, b = small
    tb, ta, tbm = _cuda(beta), _cuda(a), _cuda(b)

    def call():
        if kind in ("fp64", "fp64s"):
            return W.wigner_conv_sum(tb, ta, tbm, form=kind)
        if kind == "full":
            return W.wigner_conv_sum_full(tb, ta, tbm)
        return W.wigner_conv_sum_lmin(tb, ta, tbm, 5.0)

    assert W.wigner_device_status() == 0
    old = W.debug_set_wait_tries(0)
    try:
        C = call()
        rc = W.wigner_device_status()
    finally:
        W.debug_set_wait_tries(old)
    assert rc == WG_ERR_TIMEOUT
    C = C.cpu().numpy()
    if kind == "lmin":  # chains cut whole are written as 0 by CTAs that never wait
        assert np.all(np.isnan(C) | (C == 0))
        assert np.isnan(C).any()
    else:
        assert np.all(np.isnan(C))
    # the context is intact: the same call with the default limit matches the oracle
    C = call().cpu().numpy()
    assert W.wigner_device_status() == 0
    if kind in ("fp64", "fp64s"):
        ref = O.conv_sum(L, MB, MS, beta, a, b)
    elif kind == "full":
        ref = O.conv_sum_full(L, MB, MS, beta, a, b)
    else:
        ref = O.conv_sum(L, MB, MS, beta, a, b, offset=5.0)
    assert float(np.max(np.abs(C - ref))) <= 1e-11


_ALLOC_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1002_1050_gb300 import wigner as W, inputs as I
from oracle import oracle as O
L, MB, MS, NB = 40, 2, 40, 50
beta = I.beta_gauss_legendre(NB)[0]; a = I.sky_alm(L, MS, 1); b = I.beam_blm(L, MB, fwhm=0.1)
tb, ta, tbm = (torch.from_numpy(x).cuda() for x in (beta, a, b))
torch.cuda.synchronize()
out = []
# the first call on the device allocates the status word and the tables: both fail in turn
W.debug_inject_alloc_failures(1)
try:
    W.wigner_conv_sum(tb, ta, tbm); out.append('no error')
except W.WignerError as e:
    out.append(e.code)
W.debug_inject_alloc_failures(1)
try:
    W.wigner_conv_sum(tb, ta, tbm); out.append('no error')
except W.WignerError as e:
    out.append(e.code)
C = W.wigner_conv_sum(tb, ta, tbm).cpu().numpy()  # retry: allocates and computes
out.append(float(np.max(np.abs(C - O.conv_sum(L, MB, MS, beta, a, b)))))
# the FP32 form's stream-ordered scratch (its weight scales)
W.debug_inject_alloc_failures(1)
try:
    W.wigner_conv_sum(tb, ta, tbm, form='fp32x'); out.append('no error')
except W.WignerError as e:
    out.append(e.code)
C = W.wigner_conv_sum(tb, ta, tbm, form='fp32x').cpu().numpy()
ref = O.conv_sum(L, MB, MS, beta, a, b)
out.append(float(np.linalg.norm((C - ref).ravel()) / np.linalg.norm(ref.ravel())))
# the adjoint's workspace
G = torch.ones((MB + 1, MS + 1, NB), dtype=torch.complex128, device='cuda')
Ct = W.wigner_conv_sum(tb, ta, tbm)
W.debug_inject_alloc_failures(1)
try:
    W.wigner_conv_sum_backward(tb, ta, tbm, Ct, G); out.append('no error')
except W.WignerError as e:
    out.append(e.code)
W.wigner_conv_sum_backward(tb, ta, tbm, Ct, G)
out.append(W.wigner_device_status())
print('RESULT', out)
"""


def test_injected_allocation_failures_fresh_process(W):
    r = subprocess.run([sys.executable, "-c", _ALLOC_CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT")][-1]
    res = eval(line[len("RESULT"):])
    assert res[0] == WG_ERR_ALLOC and res[1] == WG_ERR_ALLOC, res
    assert res[2] <= 1e-11, res
    assert res[3] == WG_ERR_ALLOC and res[4] <= 1e-4, res
    assert res[5] == WG_ERR_ALLOC and res[6] == 0, res


SENT = 1.2345678e300  # a value no kernel writes


def _guarded(shape, dtype, n_guard=256):
    """A buffer of n_guard sentinel elements, the output (shape), n_guard sentinels."""
    n = int(np.prod(shape))
    flat = torch.empty((n + 2 * n_guard,), dtype=dtype, device="cuda")
    flat.fill_(complex(SENT, -SENT) if dtype == torch.complex128 else SENT)
    return flat, flat[n_guard:n_guard + n].view(shape), n_guard


def _assert_guards(flat, n_guard, n):
    head, tail = flat[:n_guard].cpu(), flat[n_guard + n:].cpu()
    if flat.dtype == torch.complex128:
        want = complex(SENT, -SENT)
        assert bool(torch.all(head == want)) and bool(torch.all(tail == want))
    else:
        assert bool(torch.all(head == SENT)) and bool(torch.all(tail == SENT))


def test_guard_words_around_outputs(W):
    L, MB, MS, NB = 160, 3, 150, 333
    g = I.beta_gauss_legendre(NB)[0]
    beta = g.copy()
    h = NB // 2
    beta[NB - h:] = math.pi - g[:h][::-1]  # exactly mirror-symmetric (the full sum requires it)
    beta[h] = math.pi / 2
    a = I.sky_alm(L, MS, 7)
    b = I.beam_blm(L, MB, fwhm=0.05)
    tb, ta, tbm = _cuda(beta), _cuda(a), _cuda(b)
    ref = O.conv_sum(L, MB, MS, beta, a, b)
    for form in ("fp64", "fp64s", "fp32x"):
        flat, out, ng = _guarded((MB + 1, MS + 1, NB), torch.complex128)
        W.wigner_conv_sum(tb, ta, tbm, form=form, out=out)
        W.check_device_status()
        _assert_guards(flat, ng, out.numel())
        err = float(np.max(np.abs(out.cpu().numpy() - ref)))
        assert err <= (1e-11 if form != "fp32x" else 1e-4 * float(np.max(np.abs(ref)))), (form, err)
    # every sky order: mirrored stores at N-1-j into the columns -m_sky
    flat, cf, ng = _guarded((MB + 1, 2 * MS + 1, NB), torch.complex128)
    W.wigner_conv_sum_full(tb, ta, tbm, out=cf)
    W.check_device_status()
    _assert_guards(flat, ng, cf.numel())
    assert float(np.max(np.abs(cf.cpu().numpy() - O.conv_sum_full(L, MB, MS, beta, a, b)))) <= 1e-11
    # the data cube: scatter into the half spectrum, cuFFT, real cube
    na, ng_ = W.fft_size(2 * MB + 1), W.fft_size(2 * MS + 1)
    flat_c, cube, ngc = _guarded((NB, na, ng_), torch.float64)
    W.wigner_data_cube(cf, na, ng_, out=cube)
    W.check_device_status()
    _assert_guards(flat_c, ngc, cube.numel())
    assert bool(torch.isfinite(cube).all())
    # the d-table and the several-column sum
    flat_d, d, ngd = _guarded((MB + 1, 41, 41, NB), torch.float64)
    W.wigner_d_table(tb, 40, MB, 40, out=d)
    W.check_device_status()
    _assert_guards(flat_d, ngd, d.numel())
    a3 = I.mc_skies(L, MS, 3, 20)
    flat_m, cm, ngm = _guarded((3, MB + 1, MS + 1, NB), torch.complex128)
    W.wigner_conv_sum_multi(tb, _cuda(a3), tbm, out=cm)
    W.check_device_status()
    _assert_guards(flat_m, ngm, cm.numel())
