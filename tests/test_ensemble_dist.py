"""Multi-GPU data path on CPU ranks (gloo, world size 2): each rank evaluates
its shard of the noise ensemble (here with the oracle, standing in for its
GPU), the shards' noise equals the global draw, and one all-reduce gives the
single-device ensemble result."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import noise, robust
from paper_2603_03639_gb300.ensemble import allreduce_mean, shard_seed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.WORKLOADS["x8"].replace(N=5, K=3, M=2, P=1, chi=4)
    prob = synth.make_problem(w)
    seed = shard_seed(w.seed_J, rank, w.M, w.N, w.noise_dist)
    J = noise.sample_J(seed, w.M, w.N, w.noise_dist, w.noise_scale)
    F, g, _ = robust.ensemble(robust.from_workload(prob, J))
    Ft = torch.tensor([F], dtype=torch.float64)
    gt = torch.tensor(g, dtype=torch.float64)
    allreduce_mean(Ft, gt)
    out[rank] = (float(Ft.item()), gt.numpy().copy(), J)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dist_kind", [0, 1])
@pytest.mark.parametrize("terms", [1, 3])
def test_shard_seeds_reproduce_the_global_noise(dist_kind, terms):
    N, M_local, R = 6, 3, 4
    J_global = noise.sample_J(99, M_local * R, N, dist_kind, 0.1, terms=terms)
    parts = [noise.sample_J(shard_seed(99, r, M_local, N, dist_kind, terms), M_local, N, dist_kind, 0.1, terms=terms)
             for r in range(R)]
    assert np.array_equal(np.concatenate(parts), J_global)


def test_two_rank_allreduce_equals_single_device_ensemble():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    w = synth.WORKLOADS["x8"].replace(N=5, K=3, M=4, P=1, chi=4)
    prob = synth.make_problem(w)
    J = noise.sample_J(w.seed_J, w.M, w.N, w.noise_dist, w.noise_scale)
    F, g, _ = robust.ensemble(robust.from_workload(prob, J))
    for r in range(2):
        Fr, gr, Jr = out[r]
        assert np.array_equal(Jr, J[2 * r: 2 * r + 2])
        assert abs(Fr - F) < 1e-15
        assert np.max(np.abs(gr - g)) < 1e-15
