"""Batched uneven instances in one persistent launch (work queue, autotuner, CUDA graph).

Each instance's output must match the single-instance entry point of its form (FP64:
1e-11 absolute; FP32 form: 1e-4 relative L2) -- run without a graph, with a graph
(first call captures, second replays, after the inputs change in place), and with the
autotuned variant.
"""
import numpy as np
import pytest
import torch

from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_1002_1050_gb300 import wigner
    wigner.load()
    return wigner


@pytest.fixture(scope="module")
def batch(W):
    specs = I.batch_instances(n=14, seed=3, l_range=(8, 420), nb_range=(1, 700))
    for i, sp in enumerate(specs):  # every third FP64 instance uses the split-pipe FP64 form
        if sp["form"] == 0 and i % 3 == 0:
            sp["form"] = 2
    a_full = torch.from_numpy(specs[0]["a_full"]).cuda()
    probs = []
    for sp in specs:
        L, MB = sp["l_max"], sp["mb_max"]
        a = a_full[:L + 1, :L + 1].contiguous()
        b = torch.from_numpy(I.beam_blm(L, MB, fwhm=0.05)).cuda()
        beta = torch.from_numpy(sp["beta"]).cuda()
        probs.append((beta, a, b, sp["form"]))
    refs = [W.wigner_conv_sum(beta, a, b, form=f) for beta, a, b, f in probs]
    W.check_device_status()
    return probs, refs


def _check(outs, probs, refs):
    for (beta, a, b, f), out, ref in zip(probs, outs, refs):
        if f in (0, 2):
            assert float((out - ref).abs().max()) <= 1e-11
        else:
            rel = float(torch.linalg.vector_norm(out - ref) / max(float(torch.linalg.vector_norm(ref)), 1e-300))
            assert rel <= 1e-4


def test_batched_convenience(W, batch):
    probs, refs = batch
    outs = W.wigner_conv_sum_batched([(beta, a, b, f, None) for beta, a, b, f in probs])
    W.check_device_status()
    _check(outs, probs, refs)
    assert {f for *_, f in probs} == {0, 1, 2}  # the batch mixes all three forms


def test_plan_graph_replay(W, batch):
    probs, refs = batch
    plan = W.BatchPlan([(beta, a, b, f, None) for beta, a, b, f in probs])
    info = plan.info()
    assert info["n_items"] > 0 and info["grid"] >= 152
    outs = plan.run(use_graph=True)
    torch.cuda.synchronize()
    _check(outs, probs, refs)
    for o in outs:
        o.zero_()
    outs = plan.run(use_graph=True)  # replay
    torch.cuda.synchronize()
    _check(outs, probs, refs)
    # inputs changed in place: the replayed graph reads the new values
    beta0, a0, b0, f0 = probs[0]
    b0.mul_(2.0)
    outs = plan.run(use_graph=True)
    torch.cuda.synchronize()
    ref0 = W.wigner_conv_sum(beta0, a0, b0, form=f0)
    b0.mul_(0.5)
    tol = 1e-11 if f0 in (0, 2) else 1e-4 * float(torch.linalg.vector_norm(ref0))
    assert float((outs[0] - ref0).abs().max()) <= tol
    plan.close()
    W.check_device_status()


def test_plan_autotune(W, batch, tmp_path, monkeypatch):
    probs, refs = batch
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("WIGNER_TUNE_CACHE", str(cache))
    plan = W.BatchPlan([(beta, a, b, f, None) for beta, a, b, f in probs], autotune=True)
    outs = plan.run()
    torch.cuda.synchronize()
    _check(outs, probs, refs)
    assert 0 <= plan.info()["variant"] < 4
    plan.close()


def test_empty_and_bad_instances(W):
    assert W.wigner_conv_sum_batched([]) == []
    beta = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    a = torch.zeros((3, 3), dtype=torch.complex128, device="cuda")
    b = torch.zeros((3, 5), dtype=torch.complex128, device="cuda")  # mb_max 4 > l_max 2
    with pytest.raises(W.WignerError):
        W.wigner_conv_sum_batched([(beta, a, b, 0, None)])
