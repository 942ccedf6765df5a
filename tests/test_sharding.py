"""Replica sharding across ranks: disjoint noise ranges and an order-fixed merge (CPU, gloo, world 2)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1012_5168_gb300 import sharding


def test_index_ranges_partition():
    for total in (0, 1, 7, 64, 1536):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                f, n = sharding.index_range(r, world, total)
                seen.extend(range(f, f + n))
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        sharding.index_range(2, 2, 5)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synthetic
    from oracle import loops, noise
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, 0.5, 3)
    minv = np.linalg.inv(__import__("oracle").wilson.dense_matrix(U, 0.12, -1.0))
    first, n = sharding.index_range(rank, world, 7)
    eta = noise.make_sources(dims, 5, first, n, noise.SPIN | noise.TIME, t0=-1)
    phi = (minv @ eta.reshape(len(eta), -1).T).T.reshape(eta.shape)
    lo = loops.stochastic_loops(eta, phi).reshape(n, 4, 16, dims[3]).sum(1)  # per noise vector
    merged = sharding.gather_to_root(lo)
    if rank == 0:
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_process(tmp_path):
    out = str(tmp_path / "merged.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    merged = np.load(out)
    import synthetic
    from oracle import loops, noise, wilson
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, 0.5, 3)
    minv = np.linalg.inv(wilson.dense_matrix(U, 0.12, -1.0))
    eta = noise.make_sources(dims, 5, 0, 7, noise.SPIN | noise.TIME, t0=-1)
    phi = (minv @ eta.reshape(len(eta), -1).T).T.reshape(eta.shape)
    ref = loops.stochastic_loops(eta, phi).reshape(7, 4, 16, dims[3]).sum(1)
    assert merged.shape == ref.shape
    assert np.allclose(merged, ref, rtol=1e-13, atol=1e-13)
