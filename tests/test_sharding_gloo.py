"""Source sharding over two CPU ranks (gloo): the shards partition the source
list, and the sum of the per-shard partial BC vectors (computed here by the
oracle on the CPU) reduced onto rank 0 equals BC over the whole list."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import bcgen
import oracle
from paper_1409_7764_gb300.sharding import reduce_partial_bc, shard_sources


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = bcgen.rmat(8, 8, seed=2)
    srcs = bcgen.sample_sources(g.n, 101, seed=4)
    mine = shard_sources(srcs, world, rank)
    part, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, mine)
    t = torch.from_numpy(part.copy())
    reduce_partial_bc(t, dist, dst=0)
    if rank == 0:
        np.save(result_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shards_partition_the_sources():
    srcs = np.arange(103, dtype=np.int32)
    parts = [shard_sources(srcs, 4, r) for r in range(4)]
    assert np.array_equal(np.concatenate(parts), srcs)
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        shard_sources(srcs, 2, 2)


def test_two_rank_reduce_equals_whole(tmp_path):
    port = _free_port()
    out = str(tmp_path / "bc.npy")
    tmp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True,
                        start_method="spawn")
    got = np.load(out)
    g = bcgen.rmat(8, 8, seed=2)
    srcs = bcgen.sample_sources(g.n, 101, seed=4)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-12)
