"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times (the batch width the library keeps for the graph after its width
trial, at most 256 sources per batch for R-MAT scale 16 exact and for 4096
sampled sources, at most 128 for 1024), on outputs the
oracle can compute: BC over source subsets run in the same configuration,
depths and path counts of single sources bit for bit, and properties of the
full runs.  Graphs and source samples are the benchmark's own (same seeds).
"""
import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu

TOL = {True: 1e-12, False: 1e-4}


@pytest.fixture(scope="module")
def ctx():
    import paper_1409_7764_gb300 as bc
    c = bc.Context(0)
    yield c
    c.close()


def close(got, ref, tol):
    zero = ref == 0
    assert np.array_equal(np.asarray(got)[zero], ref[zero]), "exact zeros differ"
    if (~zero).any():
        rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
        assert rel.max() <= tol, f"max rel err {rel.max():.3e}"


def bit_exact(ctx, G, g, srcs, kb, direction="auto"):
    d, sig, _ = ctx.debug_sources(G, np.asarray(srcs, dtype=np.int32), batch_k=kb,
                                  delta_fp64=True, direction=direction)
    for i, s in enumerate(srcs):
        od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, int(s))
        np.testing.assert_array_equal(d[i], od)
        np.testing.assert_array_equal(sig[i], osig)


def test_rmat16_exact_full_size(ctx):
    g = bcgen.rmat(16, 16, seed=1)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ctx.exact(G)                                     # first job: width and split trials
    full = ctx.exact(G).copy()                       # the benchmark's call (FP32 dependencies)
    st = ctx.last_stats()
    kb = st["batch_sources"]
    assert st["sources"] == g.n and kb in (64, 128, 256)
    # the exact result is the sum over any partition of the sources
    parts = np.array_split(np.arange(g.n, dtype=np.int32), 4)
    summed = sum(ctx.sources(G, p_, batch_k=kb).copy() for p_ in parts)
    close(full, summed, 1e-4)
    assert np.all(full >= 0)
    # 256 sources in the same configuration, element by element against the oracle
    src = bcgen.sample_sources(g.n, 256, seed=7)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, src)
    for fp64 in (False, True):
        close(ctx.sources(G, src, batch_k=kb, delta_fp64=fp64), ref, TOL[fp64])
    bit_exact(ctx, G, g, src[:6], kb)
    ctx.destroy_graph(G)


def test_rmat20_sampled_full_size(ctx):
    g = bcgen.rmat(20, 16, seed=1)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    src1024 = bcgen.sample_sources(g.n, 1024, seed=1)  # the benchmark's sources
    sub = src1024[:64]
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, sub)
    for kb in (128, 256):                              # the 1024- and 4096-source widths
        for fp64 in (False, True):
            close(ctx.sources(G, sub, batch_k=kb, delta_fp64=fp64), ref, TOL[fp64])
    # path counts pushed at every level (64-bit integer atomics) or pulled
    for direction in ("push", "pull"):
        close(ctx.sources(G, sub, batch_k=256, direction=direction), ref, TOL[False])
    bit_exact(ctx, G, g, sub[:3], 128)
    bit_exact(ctx, G, g, sub[3:5], 128, direction="push")
    # the full 1024-source job as timed: width 128, and the sum over its batches
    full = ctx.sources(G, src1024).copy()
    kb = ctx.last_stats()["batch_sources"]
    assert kb in (64, 128)
    halves = ctx.sources(G, src1024[:512], batch_k=kb) + ctx.sources(G, src1024[512:], batch_k=kb)
    close(full, halves, 1e-4)
    ctx.destroy_graph(G)


def test_ba20_sampled_full_size(ctx):
    g = bcgen.ba_directed(1 << 20, 8, 9, 1)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    src = bcgen.sample_sources(g.n, 4096, seed=1)[:256]
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, src)
    for fp64 in (False, True):
        close(ctx.sources(G, src, batch_k=256, delta_fp64=fp64), ref, TOL[fp64])
        # the benchmark's direction rule pushes counts on this DAG
        assert ctx.last_stats()["push_levels"] > 0
    for direction in ("push", "pull"):
        close(ctx.sources(G, src, batch_k=256, direction=direction), ref, TOL[False])
        st = ctx.last_stats()
        assert (st["push_levels"] > 0) == (direction == "push")
    bit_exact(ctx, G, g, src[:3], 256)
    bit_exact(ctx, G, g, src[3:5], 256, direction="pull")
    ctx.destroy_graph(G)


def test_many_graphs_full_size_sampled(ctx):
    specs = bcgen.small_rmat_specs(10000, master_seed=1)  # the benchmark's 10,000 graphs
    gs = [bcgen.rmat(s, ef, sd) for s, ef, sd in specs]
    hs = [ctx.create_graph(g.row_ptr, g.col_idx) for g in gs]
    outs = ctx.exact_many(hs)                            # one launch, FP32 dependencies
    for i in range(0, len(gs), 100):                     # every 100th graph against the oracle
        ref, _ = oracle.bc(gs[i].n, gs[i].row_ptr, gs[i].col_idx)
        close(outs[i], ref, 1e-4)
    for h in hs:
        ctx.destroy_graph(h)


def test_ba_undirected_30k_d60_full_size(ctx):
    """The paper's largest preferential-attachment input (n = 30,000, edge
    density 60: 30 undirected edges per arrival, stored both ways), exact BC
    as the benchmark runs it (256 sources per batch), checked on a 256-source
    subset in the same configuration and on properties of the full run."""
    g = bcgen.ba_undirected(30000, 30, seed=1)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ctx.exact(G)                                     # first job: width and split trials
    full = ctx.exact(G).copy()
    st = ctx.last_stats()
    kb = st["batch_sources"]
    assert st["sources"] == g.n and kb in (64, 128, 256)
    assert np.all(full >= 0)
    # every source reaches every vertex (the graph is connected)
    assert st["reached_pairs"] == g.n * g.n
    src = np.concatenate([np.arange(8), bcgen.sample_sources(g.n, 248, seed=9)]).astype(np.int32)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, src)
    for fp64 in (False, True):
        close(ctx.sources(G, src, batch_k=kb, delta_fp64=fp64), ref, TOL[fp64])
    bit_exact(ctx, G, g, src[:4], kb)
