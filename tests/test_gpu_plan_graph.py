"""Plans reserve the library's device state, after which calls within the caps allocate
nothing and can be captured into a CUDA graph (PyTorch's graph capture here)."""
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


@pytest.mark.parametrize("form,tol", [("fp64", 1e-11), ("fp64s", 1e-11), ("fp32x", None)])
def test_conv_sum_in_cuda_graph(W, form, tol):
    L, MB, MS, NB = 150, 4, 150, 300
    plan = W.Plan(l_max_cap=L, mb_max_cap=MB, ms_max_cap=MS, n_beta_cap=NB)
    beta_h = I.beta_gauss_legendre(NB)[0]
    a_h, b_h = I.sky_alm(L, MS, 2), I.beam_blm(L, MB, fwhm=0.05)
    beta, a, b = (torch.from_numpy(x).cuda() for x in (beta_h, a_h, b_h))
    out = torch.empty((MB + 1, MS + 1, NB), dtype=torch.complex128, device="cuda")
    W.wigner_conv_sum(beta, a, b, form=form, out=out)  # loads the kernel outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        W.wigner_conv_sum(beta, a, b, form=form, out=out)
    for scale in (1.0, 2.0):
        b.copy_(torch.from_numpy(b_h * scale))
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        ref = O.conv_sum(L, MB, MS, beta_h, a_h, b_h * scale)
        got = out.cpu().numpy()
        if tol is not None:
            assert np.max(np.abs(got - ref)) <= tol
        else:
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
    W.check_device_status()
    plan.close()
