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


def test_many_graphs_count_rows_and_sources_without_out_edges(ctx):
    """Path counts start in 32-bit rows: a graph whose counts reach 2^32
    (layered chains of 32 and 40 stages: 2^32 and 2^40 paths to the last
    sink) continues with 64-bit rows from the batch that found it, and every
    result equals the run with 64-bit rows throughout bit for bit and the
    oracle.  Sources without out-edges are not run: an out-star runs its
    centre alone."""
    gs = [bcgen.layered_chain(40, 2), bcgen.layered_chain(32, 2), bcgen.layered_chain(31, 2),
          bcgen.star(3000, "out"), bcgen.rmat(12, 4, seed=9), bcgen.rmat(11, 16, seed=4),
          bcgen.rmat(8, 4, seed=2)]
    handles = [ctx.create_graph(g.row_ptr, g.col_idx) for g in gs]
    for fp64, tol in ((True, 1e-12), (False, 1e-4)):
        a = [x.copy() for x in ctx.exact_many(handles, delta_fp64=fp64)]
        b = ctx.exact_many(handles, delta_fp64=fp64, count_bits=64)
        for g, x, y in zip(gs, a, b):
            np.testing.assert_array_equal(x, y)
            ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
            close(x, ref, tol)
    out = ctx.exact_many([handles[3]], delta_fp64=True)[0]
    assert ctx.last_stats()["batches"] == 1
    assert not out.any()
    # the same vectors written into a device tensor
    import torch
    host = ctx.exact_many(handles, delta_fp64=True)
    dev = torch.full((sum(g.n for g in gs),), -1.0, dtype=torch.float64, device="cuda")
    assert ctx.exact_many(handles, out=dev, delta_fp64=True) is dev
    np.testing.assert_array_equal(dev.cpu().numpy(), np.concatenate(host))
    for h in handles:
        ctx.destroy_graph(h)


def test_create_graphs_in_one_call(ctx):
    """bc_create_graphs: small graphs prepared on host threads, a large one on
    the device, a non-canonical one canonicalised; each resident graph equals
    the canonical CSR and its transpose bit for bit, BC matches the oracle,
    and one malformed graph rejects the whole call."""
    import paper_1409_7764_gb300 as bc
    rs = np.random.default_rng(2)
    src, dst = rs.integers(0, 300, 3000), rs.integers(0, 300, 3000)
    raw = bcgen.raw_csr_from_edges(300, np.concatenate([src, src[:400], np.arange(40)]),
                                   np.concatenate([dst, dst[:400], np.arange(40)]))
    canon_raw = bcgen.csr_from_edges(300, src, dst)
    gs = [bcgen.rmat(s_, ef, sd) for (s_, ef, sd) in bcgen.small_rmat_specs(300, master_seed=3)]
    gs += [bcgen.csr_from_edges(1, [], []), bcgen.star(900, "bi"), bcgen.rmat(14, 20, seed=4)]
    inputs = [(g.row_ptr, g.col_idx) for g in gs] + [(raw.row_ptr, raw.col_idx)]
    canon = gs + [canon_raw]
    hs = ctx.create_graphs(inputs)
    assert [h.m for h in hs] == [g.m for g in canon]
    for h, g in zip(hs, canon):
        rp, ci, ip, ii = ctx.debug_graph(h)
        np.testing.assert_array_equal(rp, g.row_ptr)
        np.testing.assert_array_equal(ci, g.col_idx)
        s_, d_ = g.edges()
        cnt = np.zeros(g.n + 1, dtype=np.int64)
        np.add.at(cnt, np.asarray(d_, dtype=np.int64) + 1, 1)
        np.testing.assert_array_equal(ip, np.cumsum(cnt))
        np.testing.assert_array_equal(ii, np.asarray(s_)[np.lexsort((s_, d_))])
    small = [i for i, g in enumerate(canon) if g.n <= 4096]
    outs = ctx.exact_many([hs[i] for i in small], delta_fp64=True)
    for i, got in list(zip(small, outs))[::7]:
        ref, _ = oracle.bc(canon[i].n, canon[i].row_ptr, canon[i].col_idx)
        close(got, ref, 1e-12)
    for h in hs:
        ctx.destroy_graph(h)
    bad = gs[5].col_idx.copy()
    bad[0] = gs[5].n
    with pytest.raises(bc.BCError) as ei:
        ctx.create_graphs(inputs[:5] + [(gs[5].row_ptr, bad)] + inputs[6:10])
    assert ei.value.status == bc.BC_ERR_GRAPH
    hs = ctx.create_graphs(inputs[:10])
    assert len(hs) == 10
    for h in hs:
        ctx.destroy_graph(h)
