"""Exact BC of many small graphs in one persistent launch (bc_exact_many),
against the CPU oracle graph by graph."""
import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1409_7764_gb300 as bc
    c = bc.Context(0)
    yield c
    c.close()


def close(got, ref, tol):
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero])
    if (~zero).any():
        rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
        assert rel.max() <= tol, f"max rel err {rel.max():.3e}"


def mixed_graphs():
    gs = [bcgen.rmat(s, ef, seed) for (s, ef, seed) in bcgen.small_rmat_specs(40, master_seed=7,
                                                                              scale_hi=10)]
    gs.append(bcgen.star(3001, "bi"))              # a hub split into chunks
    gs.append(bcgen.csr_from_edges(1, [], []))     # single vertex
    gs.append(bcgen.csr_from_edges(6, [], []))     # no edges
    gs.append(bcgen.path(90))                      # many levels
    gs.append(bcgen.rmat(14, 8, seed=5))           # above the per-block size: grid path
    return gs


@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-4)])
def test_many_graphs_match_oracle(ctx, fp64, tol):
    gs = mixed_graphs()
    handles = [ctx.create_graph(g.row_ptr, g.col_idx) for g in gs]
    outs = ctx.exact_many(handles, delta_fp64=fp64)
    st = ctx.last_stats()
    assert st["sources"] == sum(g.n for g in gs)
    for g, got in zip(gs, outs):
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
        close(got, ref, tol)
    for h in handles:
        ctx.destroy_graph(h)


def test_many_graphs_normalised_and_batch_width(ctx):
    gs = [bcgen.rmat(7, 6, seed=i) for i in range(5)]
    handles = [ctx.create_graph(g.row_ptr, g.col_idx) for g in gs]
    outs = ctx.exact_many(handles, delta_fp64=True, normalize=True, batch_k=23)
    for g, got in zip(gs, outs):
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
        close(got, oracle.normalise(ref, g.n), 1e-12)
    for h in handles:
        ctx.destroy_graph(h)


def test_many_graphs_per_graph_width_and_overrun(ctx):
    """Graphs of 2048+ vertices run 256 sources per batch, 1024+ run 128,
    smaller ones 64; a long path overruns a wide batch's queue in its forward
    sweep and continues 64 sources per batch.  All match the oracle."""
    gs = [bcgen.rmat(11, 8, seed=1), bcgen.rmat(10, 12, seed=2), bcgen.path(2100),
          bcgen.rmat(7, 6, seed=3), bcgen.ba_directed(2500, 4, 5, 7)]
    handles = [ctx.create_graph(g.row_ptr, g.col_idx) for g in gs]
    for fp64, tol in ((True, 1e-12), (False, 1e-4)):
        outs = ctx.exact_many(handles, delta_fp64=fp64)
        for g, got in zip(gs, outs):
            ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
            close(got, ref, tol)
    # an explicit width keeps every graph at 64 sources per batch
    outs = ctx.exact_many(handles, delta_fp64=True, batch_k=64)
    for g, got in zip(gs, outs):
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
        close(got, ref, 1e-12)
    for h in handles:
        ctx.destroy_graph(h)
