"""The multi-rank host logic on CPU (gloo, world size 2): probe shards by seed
offset reproduce the single-process probes, and the averaged per-rank energy
and force estimates equal the estimate over all probes.  The per-rank compute
is the oracle's (no GPU needed)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.forces import estimator_forces
from oracle.lanczos import rademacher_probes
from oracle.operator import Operator
from paper_2307_02278_gb300.parallel import reduce_estimates, shard_seed
from workloads.systems import random_system

R_RANK, M, SEED = 3, 10, 2307022799


def _system():
    return random_system(12, 11.0, 5, mesh=(16, 16, 16), r_cut=5.4, damp_cut=5.4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    op = Operator(_system(), "spme")
    f, e, _ = estimator_forces(op, R_RANK, M, shard_seed(SEED, rank, R_RANK))
    et = torch.tensor([e], dtype=torch.float64)
    ft = torch.tensor(f)
    reduce_estimates(et, ft)
    if rank == 0:
        out.put((float(et[0]), ft.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_seed_reproduces_global_probes():
    dim = 50
    full = rademacher_probes(SEED, 4 * R_RANK, dim)
    for rank in range(4):
        np.testing.assert_array_equal(rademacher_probes(shard_seed(SEED, rank, R_RANK), R_RANK, dim),
                                      full[rank * R_RANK:(rank + 1) * R_RANK])


@pytest.mark.timeout(300)
def test_two_rank_reduction_equals_single_process():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    e_red, f_red = out.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f_all, e_all, _ = estimator_forces(Operator(_system(), "spme"), 2 * R_RANK, M, SEED)
    assert abs(e_red - e_all) <= 1e-13 * abs(e_all)
    np.testing.assert_allclose(f_red, f_all, rtol=0, atol=1e-14 * np.abs(f_all).max())
