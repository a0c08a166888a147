"""wigner_conv_sum_host: the fused sum on host buffers, computed in blocks of sky orders
whose downloads overlap the next block's computation.  Every column is computed by the
same kernel code as in wigner_conv_sum, so the results must be identical bit for bit;
the oracle checks the values."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import wigner
    wigner.load()
    return wigner


@pytest.mark.parametrize("blocks", ["1", "4"])
@pytest.mark.parametrize("form", ["fp64", "fp64s", "fp32x"])
@pytest.mark.parametrize("L,MB,MS,NB", [(150, 4, 150, 300), (0, 0, 0, 1), (40, 3, 0, 7), (300, 8, 5, 513)])
def test_host_matches_device_and_oracle(W, form, L, MB, MS, NB, blocks, monkeypatch):
    monkeypatch.setenv("WIGNER_HOST_BLOCKS", blocks)  # 4: downloads overlap the next block
    beta = I.beta_gauss_legendre(NB)[0]
    a = I.sky_alm(L, MS, 21)
    b = I.beam_blm(L, MB, fwhm=0.05)
    pinned = [torch.from_numpy(x).pin_memory() for x in (beta, a, b)]
    C_host = W.wigner_conv_sum_host(*pinned, form=form)
    C_dev = W.wigner_conv_sum(*(x.cuda() for x in pinned), form=form).cpu()
    W.check_device_status()
    assert torch.equal(C_host, C_dev)
    ref = O.conv_sum(L, MB, MS, beta, a, b)
    got = C_host.numpy()
    if form == "fp32x":
        assert np.linalg.norm(got - ref) <= 1e-4 * max(np.linalg.norm(ref), 1e-300)
    else:
        assert np.max(np.abs(got - ref)) <= 1e-11


def test_host_pageable_buffers(W):
    """numpy (pageable) inputs and output work too (copied synchronously)."""
    L, MB, MS, NB = 90, 2, 90, 65
    beta = I.beta_uniform(NB, 0.02, math.pi - 0.02, 22)
    a = I.sky_alm(L, MS, 23)
    b = I.beam_blm(L, MB, fwhm=0.05)
    out = torch.empty((MB + 1, MS + 1, NB), dtype=torch.complex128)
    W.wigner_conv_sum_host(beta, a, b, out=out)
    assert np.max(np.abs(out.numpy() - O.conv_sum(L, MB, MS, beta, a, b))) <= 1e-11
