"""Angle sharding over ranks, on CPU with the gloo backend (world size 2).

Each rank takes its block of angles from `angle_shard`, computes the oracle's C and
gradients for that block, and the gradients with respect to the replicated a and b
are summed with `allreduce_sum_`.  The concatenated C and the all-reduced gradients
must equal the unsharded computation; grad_beta stays local to each rank's angles.
(The GPU kernels are not needed for this host-side logic.)
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1002_1050_gb300.distributed import allreduce_sum_, angle_shard


def test_angle_shard_partitions():
    for n in (0, 1, 7, 64, 2048):
        for world in (1, 2, 3, 8):
            sl = [angle_shard(n, r, world) for r in range(world)]
            idx = np.concatenate([np.arange(n)[s] for s in sl]) if n else np.array([])
            assert np.array_equal(idx, np.arange(n))
            sizes = [s.stop - s.start for s in sl]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import oracle as O
    from paper_1002_1050_gb300 import inputs as I

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, MB, MS, NB = 20, 2, 20, 11
    beta = I.beta_uniform(NB, 0.05, math.pi - 0.05, 3)
    a = I.sky_alm(L, MS, 1)
    b = I.beam_blm(L, MB, fwhm=0.3)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((MB + 1, MS + 1, NB)) + 1j * rng.standard_normal((MB + 1, MS + 1, NB))
    sl = angle_shard(NB, rank, world)
    C_loc = O.conv_sum(L, MB, MS, beta[sl], a, b)
    ga, gb, gbeta = O.conv_grad(L, MB, MS, beta[sl], a, b, np.ascontiguousarray(G[:, :, sl]))
    ta, tb = torch.from_numpy(ga), torch.from_numpy(gb)
    allreduce_sum_(ta, tb)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), C=C_loc, ga=ta.numpy(), gb=tb.numpy(), gbeta=gbeta,
             start=sl.start, stop=sl.stop)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_gradients_match_unsharded(tmp_path):
    from oracle import oracle as O
    from paper_1002_1050_gb300 import inputs as I

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    L, MB, MS, NB = 20, 2, 20, 11
    beta = I.beta_uniform(NB, 0.05, math.pi - 0.05, 3)
    a = I.sky_alm(L, MS, 1)
    b = I.beam_blm(L, MB, fwhm=0.3)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((MB + 1, MS + 1, NB)) + 1j * rng.standard_normal((MB + 1, MS + 1, NB))
    C = O.conv_sum(L, MB, MS, beta, a, b)
    ga, gb, gbeta = O.conv_grad(L, MB, MS, beta, a, b, G)
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    C_sh = np.concatenate([p["C"] for p in parts], axis=2)
    np.testing.assert_allclose(C_sh, C, rtol=0, atol=1e-15)
    for p in parts:  # every rank holds the full-job gradient w.r.t. the replicated inputs
        np.testing.assert_allclose(p["ga"], ga, rtol=0, atol=1e-13)
        np.testing.assert_allclose(p["gb"], gb, rtol=0, atol=1e-13)
    gbeta_sh = np.concatenate([p["gbeta"] for p in parts])
    np.testing.assert_allclose(gbeta_sh, gbeta, rtol=0, atol=1e-13)
