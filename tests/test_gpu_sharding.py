"""The sharded library path: two ranks (gloo, spawned processes) share cuda:0,
each computes its contiguous shard of the source list through the C ABI
(bc_sources), and the partial BC vectors are summed onto rank 0 with the
process group's reduce, the method's one exchange step.  The sum must equal
the oracle over the whole list.  The ranks' kernels never wait on each other:
each launch synchronises only its own thread blocks."""
import os
import socket

import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graph():
    return bcgen.rmat(11, 8, seed=6)


def _sources(g):
    return bcgen.sample_sources(g.n, 301, seed=9)


def _worker(rank, world, port, result_path, fp64):
    import torch
    import torch.distributed as dist
    import paper_1409_7764_gb300 as bc
    from paper_1409_7764_gb300.sharding import reduce_partial_bc, shard_sources
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = _graph()
    mine = shard_sources(_sources(g), world, rank)
    with bc.Context(0) as ctx:
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        part = ctx.sources(G, mine, delta_fp64=fp64).copy()
        ctx.destroy_graph(G)
    t = torch.from_numpy(part)
    reduce_partial_bc(t, dist, dst=0)
    if rank == 0:
        np.save(result_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("fp64", [True, False])
def test_two_rank_library_shards_sum_to_the_whole(tmp_path, fp64):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    out = str(tmp_path / "bc.npy")
    tmp.start_processes(_worker, args=(2, _free_port(), out, fp64), nprocs=2, join=True,
                        start_method="spawn")
    got = np.load(out)
    g = _graph()
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, _sources(g))
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero])
    rel = np.abs(got[~zero] - ref[~zero]) / ref[~zero]
    assert rel.max() <= (1e-12 if fp64 else 1e-4)
