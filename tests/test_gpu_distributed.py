"""The angle-sharded product path, ShardedConvSum, run by two gloo ranks that share this
process's GPU (the kernels of the two ranks never wait on each other: the only exchange
is the host-side all-reduce of grad_a and grad_b in the backward pass).

Each rank computes C for its contiguous block of angles (`angle_shard`), a squared-error
loss against a seeded target, and calls backward.  The concatenated C must equal the
oracle's sum over the whole angle set, each rank's grad_a and grad_b (all-reduced) the
oracle's whole-job gradients, and the concatenated grad_beta the oracle's -- the
beta-subset distribution of Sec. 4.1.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1002_1050_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L, MB, MS, NB = 120, 4, 100, 301


def _problem():
    beta = I.beta_uniform(NB, 0.02, math.pi - 0.02, 9)
    a = I.sky_alm(L, MS, 3)
    rng = np.random.default_rng(4)
    b = I.beam_blm(L, MB, fwhm=0.05) + 0.05j * rng.standard_normal((L + 1, MB + 1))
    b[np.arange(MB + 1)[None, :] > np.arange(L + 1)[:, None]] = 0
    T = rng.standard_normal((MB + 1, MS + 1, NB)) + 1j * rng.standard_normal((MB + 1, MS + 1, NB))
    return beta, a, np.ascontiguousarray(b), 1e-3 * T


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    from paper_1002_1050_gb300 import wigner as W
    from paper_1002_1050_gb300.distributed import ShardedConvSum, angle_shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W.load()
    beta, a, b, T = _problem()
    sl = angle_shard(NB, rank, world)
    ta = torch.from_numpy(a).cuda().requires_grad_(True)
    tb = torch.from_numpy(b).cuda().requires_grad_(True)
    tbeta = torch.from_numpy(np.ascontiguousarray(beta[sl])).cuda().requires_grad_(True)
    tT = torch.from_numpy(np.ascontiguousarray(T[:, :, sl])).cuda()
    C = ShardedConvSum.apply(ta, tb, tbeta)
    loss = torch.sum(torch.abs(C - tT) ** 2)
    loss.backward()
    torch.cuda.synchronize()
    W.check_device_status()
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), C=C.detach().cpu().numpy(), ga=ta.grad.cpu().numpy(),
             gb=tb.grad.cpu().numpy(), gbeta=tbeta.grad.cpu().numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_conv_sum_two_ranks_match_oracle(tmp_path):
    import __graft_entry__ as g
    g.build()
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    beta, a, b, T = _problem()
    C = O.conv_sum(L, MB, MS, beta, a, b)
    ga, gb, gbeta = O.conv_grad(L, MB, MS, beta, a, b, 2.0 * (C - T))
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    assert np.max(np.abs(np.concatenate([p["C"] for p in parts], axis=2) - C)) <= 1e-11
    for p in parts:  # both ranks hold the whole job's gradient of the replicated inputs
        for got, ref in ((p["ga"], ga), (p["gb"], gb)):
            assert np.max(np.abs(got - ref)) <= 1e-10 * max(1.0, float(np.max(np.abs(ref))))
    gbeta_sh = np.concatenate([p["gbeta"] for p in parts])
    assert np.max(np.abs(gbeta_sh - gbeta)) <= 1e-10 * max(1.0, float(np.max(np.abs(gbeta))))
