"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars:
  * depths d[] and path counts sigma[]: bit-exact (integers);
  * BC: where the oracle gives exactly 0 the GPU must give exactly 0;
    elsewhere relative error <= 1e-12 with FP64 dependencies and <= 1e-4 with
    FP32 dependencies.  Every term of the dependency sums is positive (no
    cancellation), so each value carries a few ulps per level and per summed
    term: with levels x log2(degree) x a few <= 10^3 that stays near 1e-13
    in FP64 (eps 1.1e-16) and near 1e-5 in FP32 (eps 6e-8).
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


def assert_bc_close(got, ref, fp64):
    got = np.asarray(got)
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero]), "exact zeros differ"
    nz = ~zero
    if nz.any():
        rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
        assert rel.max() <= TOL[fp64], f"max rel err {rel.max():.3e}"


def graphs_small():
    return [
        bcgen.path(37), bcgen.path(16, bidirected=True), bcgen.cycle(21), bcgen.star(40, "bi"),
        bcgen.star(30, "out"), bcgen.complete(9), bcgen.grid(6, 7), bcgen.rmat(8, 8, seed=1),
        bcgen.rmat(10, 8, seed=1), bcgen.ba_directed(700, 4, 5, seed=2),
        bcgen.random_digraph(50, 0.08, 3), bcgen.ba_undirected(600, 3, seed=2),
        bcgen.ba_undirected(400, 1, seed=3),
    ]


def hub_graph():
    """A bidirected star with 3000 leaves (in+out degree 6000 at the hub, so
    it is split into many chunks), a 40-vertex path hanging off a leaf
    (many levels) and random extra edges."""
    n_leaf = 3000
    hub = 0
    leaves = np.arange(1, n_leaf + 1)
    tail = np.arange(n_leaf + 1, n_leaf + 41)
    src = [np.zeros(n_leaf, int), leaves, [5], tail[:-1]]
    dst = [leaves, np.zeros(n_leaf, int), [tail[0]], tail[1:]]
    rs = np.random.default_rng(4)
    extra_s = rs.integers(0, n_leaf + 41, 2000)
    extra_d = rs.integers(0, n_leaf + 41, 2000)
    src = np.concatenate([np.concatenate([np.asarray(x) for x in src]), extra_s])
    dst = np.concatenate([np.concatenate([np.asarray(x) for x in dst]), extra_d])
    return bcgen.csr_from_edges(n_leaf + 41, src, dst, name="hub+tail")


@pytest.mark.parametrize("schedule", ["plain", "batch"])
@pytest.mark.parametrize("fp64", [True, False])
def test_exact_bc_small_graphs(ctx, schedule, fp64):
    for g in graphs_small():
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
        got = ctx.exact(G, schedule=schedule, delta_fp64=fp64)
        assert_bc_close(got, ref, fp64)
        ctx.destroy_graph(G)


@pytest.mark.parametrize("schedule", ["plain", "batch"])
def test_depth_and_counts_bit_exact(ctx, schedule):
    g = bcgen.rmat(10, 8, seed=1)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    srcs = bcgen.sample_sources(g.n, 100, seed=7)  # 64 + ragged 36
    d, sig, dl = ctx.debug_sources(G, srcs, schedule=schedule, delta_fp64=True)
    for j, s in enumerate(srcs):
        od, osig, odl, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, int(s))
        np.testing.assert_array_equal(d[j], od)
        np.testing.assert_array_equal(sig[j], osig)
        nz = odl != 0
        assert np.array_equal(dl[j][~nz], odl[~nz])
        np.testing.assert_allclose(dl[j][nz], odl[nz], rtol=1e-12, atol=0)
    ctx.destroy_graph(G)


@pytest.mark.parametrize("schedule", ["plain", "batch"])
def test_high_degree_chunks(ctx, schedule):
    g = hub_graph()
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    srcs = np.array([0, 1, 2, 3000, 5, 3001, 17, 0], dtype=np.int32)  # hub twice
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    got = ctx.sources(G, srcs, schedule=schedule, delta_fp64=True)
    assert_bc_close(got, ref, True)
    assert ctx.last_stats()["heavy_chunks"] > 0
    d, sig, _ = ctx.debug_sources(G, srcs[:3], schedule=schedule, delta_fp64=True)
    for j, s in enumerate(srcs[:3]):
        od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, int(s))
        np.testing.assert_array_equal(d[j], od)
        np.testing.assert_array_equal(sig[j], osig)
    ref_all, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    assert_bc_close(ctx.exact(G, schedule=schedule, delta_fp64=True), ref_all, True)
    ctx.destroy_graph(G)


@pytest.mark.parametrize("schedule", ["plain", "batch"])
def test_sigma_overflow(ctx, schedule):
    import paper_1409_7764_gb300 as bc
    ok = bcgen.layered_chain(63, 2)
    G = ctx.create_graph(ok.row_ptr, ok.col_idx)
    d, sig, _ = ctx.debug_sources(G, [0], schedule=schedule, delta_fp64=True)
    assert int(sig[0][ok.n - 1]) == 2 ** 63
    ctx.destroy_graph(G)
    bad = bcgen.layered_chain(64, 2)
    G = ctx.create_graph(bad.row_ptr, bad.col_idx)
    with pytest.raises(bc.BCError) as ei:
        ctx.sources(G, [0, 1], schedule=schedule)
    assert ei.value.status == bc.BC_ERR_SIGMA_OVERFLOW
    assert ei.value.stats["overflow_sources"] == 1
    assert ctx.last_overflow_sources().tolist() == [0]
    # saturated counts still match the oracle's saturating counts bit for bit
    d, sig, _ = ctx.debug_sources(G, [0], schedule=schedule, delta_fp64=True)
    od, osig, _, ovf = oracle.single_source(bad.n, bad.row_ptr, bad.col_idx, 0)
    assert ovf
    np.testing.assert_array_equal(d[0], od)
    np.testing.assert_array_equal(sig[0], osig)
    ctx.destroy_graph(G)


def test_counts_left_by_earlier_jobs_are_never_read():
    """Path counts are not reset after a batch (a count is only read where the
    same batch wrote it).  Jobs that first fill a workspace with huge counts
    (2^30 paths, 91 vertices) and then reuse it for smaller graphs whose
    counts are small still match the oracle."""
    import paper_1409_7764_gb300 as bc
    schedule = "batch"
    chain = bcgen.layered_chain(30, 2)
    others = [bcgen.rmat(6, 8, seed=2), bcgen.ba_undirected(90, 2, seed=1)]
    with bc.Context(0) as fresh:
        for g in [chain] + others + [chain]:
            G = fresh.create_graph(g.row_ptr, g.col_idx)
            ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
            assert_bc_close(fresh.exact(G, delta_fp64=True, schedule=schedule), ref, True)
            d, sig, _ = fresh.debug_sources(G, [1, 2], schedule=schedule, delta_fp64=True)
            for j, s_ in enumerate([1, 2]):
                od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, s_)
                np.testing.assert_array_equal(d[j], od)
                np.testing.assert_array_equal(sig[j], osig)
            fresh.destroy_graph(G)


@pytest.mark.parametrize("fp64", [True, False])
def test_sampled_sources_ragged_and_duplicates(ctx, fp64):
    g = bcgen.rmat(12, 16, seed=3)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    srcs = np.concatenate([bcgen.sample_sources(g.n, 150, seed=11), [3, 3, 3]]).astype(np.int32)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    got = ctx.sources(G, srcs, delta_fp64=fp64)
    assert_bc_close(got, ref, fp64)
    scaled = ctx.sources(G, srcs, delta_fp64=fp64, scale_sampled=True)
    np.testing.assert_allclose(scaled, got * g.n / len(srcs), rtol=1e-15)
    normed = ctx.sources(G, srcs, delta_fp64=fp64, normalize=True)
    np.testing.assert_allclose(normed, oracle.normalise(got, g.n), rtol=1e-15)
    ctx.destroy_graph(G)


def test_edge_cases(ctx):
    import paper_1409_7764_gb300 as bc
    # single vertex, no edges
    G = ctx.create_graph([0, 0], [])
    assert ctx.exact(G).tolist() == [0.0]
    ctx.destroy_graph(G)
    # edgeless graph
    G = ctx.create_graph([0] * 6, [])
    assert ctx.exact(G, schedule="plain").tolist() == [0.0] * 5
    assert ctx.exact(G, schedule="batch").tolist() == [0.0] * 5
    ctx.destroy_graph(G)
    # empty source list
    g = bcgen.rmat(6, 4, seed=2)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    assert not ctx.sources(G, []).any()
    with pytest.raises(bc.BCError) as ei:
        ctx.sources(G, [g.n])
    assert ei.value.status == bc.BC_ERR_ARG
    ctx.destroy_graph(G)
    # malformed CSR
    with pytest.raises(bc.BCError) as ei:
        ctx.create_graph([0, 2, 1, 2], [1, 2], n=3)
    assert ei.value.status == bc.BC_ERR_GRAPH
    with pytest.raises(bc.BCError) as ei:
        ctx.create_graph([0, 1, 1, 2], [1, 7], n=3)
    assert ei.value.status == bc.BC_ERR_GRAPH


def check_resident(ctx, G, g):
    """The graph as the library holds it equals the canonical CSR of g and
    its transpose with ascending in-rows, bit for bit."""
    rp, ci, ip, ii = ctx.debug_graph(G)
    np.testing.assert_array_equal(rp, g.row_ptr)
    np.testing.assert_array_equal(ci, g.col_idx)
    src, dst = g.edges()
    cnt = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(cnt, np.asarray(dst, dtype=np.int64) + 1, 1)
    np.testing.assert_array_equal(ip, np.cumsum(cnt))
    np.testing.assert_array_equal(ii, np.asarray(src)[np.lexsort((src, dst))])


def test_resident_graph_small_host_prepared(ctx):
    for g in (bcgen.rmat(8, 8, seed=1), bcgen.star(300, "bi"), bcgen.csr_from_edges(5, [], [])):
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        check_resident(ctx, G, g)
        ctx.destroy_graph(G)


def test_large_graphs_validated_and_canonicalised_on_the_device(ctx):
    """Graphs above 2^18 edges are prepared on the device: a column id out of
    range (past the end, or negative) is rejected, and rows with duplicates
    and self-loops are canonicalised, with the same BC as the canonical
    graph."""
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(14, 20, seed=4)
    assert g.m > 1 << 18
    for bad in (g.n, -1):
        ci = g.col_idx.copy()
        ci[g.m // 2] = bad
        with pytest.raises(bc.BCError) as ei:
            ctx.create_graph(g.row_ptr, ci)
        assert ei.value.status == bc.BC_ERR_GRAPH
    src, dst = g.edges()
    rs = np.random.default_rng(8)
    dup = rs.integers(0, g.m, 30000)
    loops = rs.integers(0, g.n, 2000)
    raw = bcgen.raw_csr_from_edges(g.n, np.concatenate([src, src[dup], loops]),
                                   np.concatenate([dst, dst[dup], loops]))
    G = ctx.create_graph(raw.row_ptr, raw.col_idx)
    assert G.m == g.m
    check_resident(ctx, G, g)
    G2 = ctx.create_graph(g.row_ptr, g.col_idx)
    check_resident(ctx, G2, g)
    ctx.destroy_graph(G2)
    srcs = bcgen.sample_sources(g.n, 300, seed=2)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    assert_bc_close(ctx.sources(G, srcs, delta_fp64=True), ref, True)
    d, sig, _ = ctx.debug_sources(G, srcs[:3], delta_fp64=True)
    for j, s_ in enumerate(srcs[:3]):
        od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, int(s_))
        np.testing.assert_array_equal(d[j], od)
        np.testing.assert_array_equal(sig[j], osig)
    ctx.destroy_graph(G)


def test_device_prepared_graph_with_long_in_rows(ctx):
    """In-rows longer than the shared-memory sort (8192 entries) are sorted in
    place on the device: a graph whose hubs have 10,000-40,000 in-edges gives
    the oracle's BC and the oracle's path counts."""
    n = 60000
    rs = np.random.default_rng(3)
    hubs = np.array([7, 500, 59999])
    src = [rs.integers(0, n, 40000), rs.integers(0, n, 10000), rs.integers(0, n, 8193),
           rs.integers(0, n, 300000)]
    dst = [np.full(40000, hubs[0]), np.full(10000, hubs[1]), np.full(8193, hubs[2]),
           rs.integers(0, n, 300000)]
    g = bcgen.csr_from_edges(n, np.concatenate(src), np.concatenate(dst), name="long-in-rows")
    assert g.m > 1 << 18
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    check_resident(ctx, G, g)
    srcs = np.concatenate([bcgen.sample_sources(n, 200, seed=4), hubs]).astype(np.int32)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    for fp64 in (True, False):
        assert_bc_close(ctx.sources(G, srcs, delta_fp64=fp64), ref, fp64)
    d, sig, _ = ctx.debug_sources(G, srcs[:4], delta_fp64=True)
    for j, s_ in enumerate(srcs[:4]):
        od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, int(s_))
        np.testing.assert_array_equal(d[j], od)
        np.testing.assert_array_equal(sig[j], osig)
    ctx.destroy_graph(G)


def test_canonicalisation_in_library(ctx):
    rs = np.random.default_rng(5)
    n = 300
    src = rs.integers(0, n, 3000)
    dst = rs.integers(0, n, 3000)
    src = np.concatenate([src, src[:500], np.arange(50)])
    dst = np.concatenate([dst, dst[:500], np.arange(50)])
    raw = bcgen.raw_csr_from_edges(n, src, dst)
    canon = bcgen.csr_from_edges(n, src, dst)
    G = ctx.create_graph(raw.row_ptr, raw.col_idx)
    assert G.m == canon.m
    ref, _ = oracle.bc(n, canon.row_ptr, canon.col_idx)
    assert_bc_close(ctx.exact(G, delta_fp64=True), ref, True)
    ctx.destroy_graph(G)


def test_deterministic_and_batch_width_independent(ctx):
    """No atomics touch a dependency: every sum runs in a fixed order (CSR
    order within an entry, chunk order across the chunks of a hub, batch
    order across batches), so a repeated job gives the same bits, and every
    batch width agrees with the oracle within the parity tolerance."""
    g = bcgen.rmat(11, 16, seed=9)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    for fp64 in (False, True):
        for sched in ("batch", "plain"):
            ctx.exact(G, delta_fp64=fp64, schedule=sched)  # settles any per-graph tuning
            a = ctx.exact(G, delta_fp64=fp64, schedule=sched).copy()
            b = ctx.exact(G, delta_fp64=fp64, schedule=sched).copy()
            assert_bc_close(a, ref, fp64)
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), f"{sched} fp64={fp64}"
    for kb in (1, 7, 32, 64, 100, 128, 200, 256):
        assert_bc_close(ctx.exact(G, delta_fp64=True, batch_k=kb), ref, True)
    ctx.destroy_graph(G)


def test_device_output(ctx):
    torch = pytest.importorskip("torch")
    g = bcgen.rmat(9, 8, seed=4)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    ctx.exact(G, out=out, delta_fp64=True)
    torch.cuda.synchronize()
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    assert_bc_close(out.cpu().numpy(), ref, True)
    ctx.destroy_graph(G)


def test_failure_injection_times_out_and_recovers(ctx):
    """One thread block skips its barrier arrival: the others give up after
    the short limit, the call reports BC_ERR_TIMEOUT, and the next call on
    the same context is correct."""
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(9, 8, seed=6)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ctx.inject_barrier_skip(1, 50)
    with pytest.raises(bc.BCError) as ei:
        ctx.exact(G, schedule="batch")
    assert ei.value.status == bc.BC_ERR_TIMEOUT
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    assert_bc_close(ctx.exact(G, schedule="batch", delta_fp64=True), ref, True)
    ctx.destroy_graph(G)


def test_deep_graph(ctx):
    """Hundreds of BFS levels (a long path with two shortcuts): one grid
    barrier per level, every level's queue segment, still exact."""
    g = bcgen.csr_from_edges(300, np.concatenate([np.arange(299), [0, 5]]),
                             np.concatenate([np.arange(1, 300), [2, 9]]), name="long path")
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    for fp64 in (True, False):
        assert_bc_close(ctx.exact(G, schedule="batch", delta_fp64=fp64), ref, fp64)
        st = ctx.last_stats()
        assert st["kernel_kind"] == 2 and st["max_levels"] > 64
    ctx.destroy_graph(G)


@pytest.mark.parametrize("schedule,kind", [("batch", 2), ("batch_queue", 2), ("plain", 1)])
def test_batched_schedules_pick_their_kernel(ctx, schedule, kind):
    g = bcgen.rmat(9, 8, seed=3)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    for fp64 in (True, False):
        assert_bc_close(ctx.exact(G, schedule=schedule, delta_fp64=fp64), ref, fp64)
        assert ctx.last_stats()["kernel_kind"] == kind
    ctx.destroy_graph(G)


@pytest.mark.parametrize("fp64", [True, False])
def test_batch_composition(ctx, fp64):
    """The library's grouping of sources into batches (default) and the given
    order compute the same BC within the parity tolerance, both against the
    oracle, for exact and sampled jobs (duplicates included); grouping shares
    frontier entries among more sources, so it needs fewer of them."""
    g = bcgen.rmat(12, 16, seed=5)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    grouped = ctx.exact(G, delta_fp64=fp64).copy()
    e_grouped = ctx.last_stats()["frontier_entries"]
    given = ctx.exact(G, delta_fp64=fp64, keep_source_order=True).copy()
    e_given = ctx.last_stats()["frontier_entries"]
    assert_bc_close(grouped, ref, fp64)
    assert_bc_close(given, ref, fp64)
    assert e_grouped < e_given
    srcs = np.concatenate([bcgen.sample_sources(g.n, 700, seed=2), [9, 9, 17]]).astype(np.int32)
    sref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    assert_bc_close(ctx.sources(G, srcs, delta_fp64=fp64), sref, fp64)
    assert_bc_close(ctx.sources(G, srcs, delta_fp64=fp64, keep_source_order=True), sref, fp64)
    assert_bc_close(ctx.sources(G, srcs[::-1].copy(), delta_fp64=fp64), sref, fp64)
    ctx.destroy_graph(G)


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("kb", [65, 128, 200, 256])
def test_wide_batches(ctx, fp64, kb):
    """Batches of more than 64 sources (masks of 2 or 4 words): exact and
    sampled BC against the oracle, including hubs split into chunks, a ragged
    last batch and duplicate sources; d and sigma stay bit-exact through the
    same kernel (checked on the narrow debug path elsewhere)."""
    g = hub_graph()
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    got = ctx.exact(G, delta_fp64=fp64, batch_k=kb, schedule="batch_queue")
    st = ctx.last_stats()
    assert st["batch_sources"] == kb and st["mask_words"] == (2 if kb <= 128 else 4)
    assert_bc_close(got, ref, fp64)
    r = bcgen.rmat(12, 16, seed=8)
    R = ctx.create_graph(r.row_ptr, r.col_idx)
    srcs = np.concatenate([bcgen.sample_sources(r.n, 900, seed=4), [5, 5, 7]]).astype(np.int32)
    sref, _ = oracle.bc(r.n, r.row_ptr, r.col_idx, srcs)
    assert_bc_close(ctx.sources(R, srcs, delta_fp64=fp64, batch_k=kb), sref, fp64)
    ctx.destroy_graph(G)
    ctx.destroy_graph(R)


def test_wide_batch_width_is_automatic(ctx):
    """Without batch_k the widest batch is 256 sources once the job has eight
    such batches, 128 below that, and 64 for small jobs; the graph's first
    job with narrower alternatives and enough sources tries them (two
    batches each) and later jobs take the fastest width, never wider than
    the rule allows."""
    g = bcgen.rmat(11, 8, seed=2)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    for k, words in ((2048, 4), (1800, 2), (1024, 2), (1000, 1), (300, 1), (2048, 4)):
        srcs = bcgen.sample_sources(g.n, k, seed=k)
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
        assert_bc_close(ctx.sources(G, srcs, delta_fp64=True), ref, True)
        assert 1 <= ctx.last_stats()["mask_words"] <= words
        if words == 1:
            assert ctx.last_stats()["mask_words"] == 1
    ctx.destroy_graph(G)


def test_wide_batch_overflow_flags(ctx):
    """Path-count overflow in a batch of 256 sources: the job reports it and
    counts the flagged sources exactly as the oracle does."""
    import paper_1409_7764_gb300 as bc
    g = bcgen.layered_chain(64, 2)  # 2^64 paths from the first vertex to the last
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    srcs = np.concatenate([np.zeros(3, np.int32), np.arange(g.n, dtype=np.int32)])
    _, ovf = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    with pytest.raises(bc.BCError) as ei:
        ctx.sources(G, srcs, batch_k=256, delta_fp64=True)
    assert ei.value.status == bc.BC_ERR_SIGMA_OVERFLOW
    assert ei.value.stats["overflow_sources"] == int(np.count_nonzero(ovf))
    assert ei.value.stats["mask_words"] == 4
    # the flagged sources, each flagged occurrence listed, as the oracle flags them
    assert ctx.last_overflow_sources().tolist() == sorted(srcs[np.nonzero(ovf)[0]].tolist())
    ctx.destroy_graph(G)


def test_wide_batch_depths_and_counts_bit_exact(ctx):
    """Depths and path counts of every source of a 256-source batch (and a
    ragged 150-source one) equal the oracle's bit for bit."""
    g = hub_graph()
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    srcs = np.concatenate([bcgen.sample_sources(g.n, 250, seed=3), [0, 0, 5, 3040, 3040, 1]])
    for kb in (256, 150):
        d, sig, dl = ctx.debug_sources(G, srcs.astype(np.int32), batch_k=kb, delta_fp64=True)
        for i, s_ in enumerate(srcs):
            od, osig, odl, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, int(s_))
            np.testing.assert_array_equal(d[i], od)
            np.testing.assert_array_equal(sig[i], osig)
            np.testing.assert_allclose(dl[i], odl, rtol=1e-12, atol=0)
    ctx.destroy_graph(G)


def test_wide_batch_queue_overrun_reruns_narrow():
    """A long path with 256 sources along it queues the deep vertices at more
    than 64 distinct depths: the wide batch overruns its queue (sized for 64
    depths per vertex; a fresh context, so no larger cached workspace), the
    job reruns with 64 sources per batch and is still exact; later jobs on the
    graph stay narrow."""
    import paper_1409_7764_gb300 as bc
    g = bcgen.path(320)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    with bc.Context(0) as fresh:
        G = fresh.create_graph(g.row_ptr, g.col_idx)
        got = fresh.exact(G, delta_fp64=True, batch_k=256, schedule="batch_queue")
        assert_bc_close(got, ref, True)
        assert fresh.last_stats()["mask_words"] == 1
        assert_bc_close(fresh.exact(G, delta_fp64=False, batch_k=256), ref, False)
        assert fresh.last_stats()["mask_words"] == 1
        fresh.destroy_graph(G)


def test_width_limits_of_other_schedules(ctx):
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(8, 8, seed=1)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    for call in (lambda: ctx.exact_many([G], batch_k=128),
                 lambda: ctx.exact(G, batch_k=257)):
        with pytest.raises(bc.BCError) as ei:
            call()
        assert ei.value.status == bc.BC_ERR_ARG
    ctx.destroy_graph(G)


@pytest.mark.parametrize("direction", ["push", "pull", "auto"])
def test_path_count_directions(ctx, direction):
    """The forward path-count step pulled over in-edges, pushed along the
    previous level's out-edges (64-bit integer atomics), or chosen per level:
    depths and counts bit for bit, BC against the oracle, on graphs with hubs
    on either side (R-MAT), a DAG whose old vertices collect huge in-degrees
    (directed preferential attachment) and an undirected one."""
    graphs = [bcgen.rmat(11, 16, seed=3), bcgen.ba_directed(3000, 8, 9, seed=2),
              bcgen.ba_undirected(1500, 6, seed=4), hub_graph()]
    for g in graphs:
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
        for fp64 in (True, False):
            for kb in (0, 64):
                got = ctx.exact(G, delta_fp64=fp64, batch_k=kb, direction=direction)
                assert_bc_close(got, ref, fp64)
                st = ctx.last_stats()
                if direction == "push":
                    assert st["push_levels"] > 0
                if direction == "pull":
                    assert st["push_levels"] == 0
        srcs = [0, 1, g.n // 2, g.n - 1]
        d, sig, _ = ctx.debug_sources(G, srcs, delta_fp64=True, direction=direction)
        for j, s_ in enumerate(srcs):
            od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, s_)
            np.testing.assert_array_equal(d[j], od)
            np.testing.assert_array_equal(sig[j], osig)
        ctx.destroy_graph(G)


def test_pushed_counts_fall_back_to_pulling_near_overflow():
    """Pushed counts of 2^32 or more could carry unseen in an atomic sum, so
    the job reruns pulling (where every add checks its carry); overflow is
    then flagged and the saturated counts match the oracle's."""
    import paper_1409_7764_gb300 as bc
    with bc.Context(0) as fresh:
        ok = bcgen.layered_chain(40, 2)  # 2^40 paths: exact, but too large to push
        G = fresh.create_graph(ok.row_ptr, ok.col_idx)
        ref, _ = oracle.bc(ok.n, ok.row_ptr, ok.col_idx)
        assert_bc_close(fresh.exact(G, delta_fp64=True, direction="push"), ref, True)
        d, sig, _ = fresh.debug_sources(G, [0], delta_fp64=True, direction="push")
        od, osig, _, _ = oracle.single_source(ok.n, ok.row_ptr, ok.col_idx, 0)
        np.testing.assert_array_equal(sig[0], osig)
        fresh.destroy_graph(G)
        bad = bcgen.layered_chain(64, 2)
        G = fresh.create_graph(bad.row_ptr, bad.col_idx)
        with pytest.raises(bc.BCError) as ei:
            fresh.sources(G, [0, 1], direction="push")
        assert ei.value.status == bc.BC_ERR_SIGMA_OVERFLOW
        d, sig, _ = fresh.debug_sources(G, [0], delta_fp64=True, direction="push")
        od, osig, _, ovf = oracle.single_source(bad.n, bad.row_ptr, bad.col_idx, 0)
        assert ovf
        np.testing.assert_array_equal(sig[0], osig)
        fresh.destroy_graph(G)


@pytest.mark.parametrize("schedule", ["batch_vertex", "batch_warp", "batch_edge", "batch", "plain"])
def test_every_schedule_and_width(ctx, schedule):
    """Every work split the tuner chooses from (vertex-centric, warp-centric
    with 256-edge hub chunks, edge-leaning 128-edge chunks), the tuned one
    and the one-source-per-launch path, at every batch width: BC against the
    oracle, and a repeated job gives the same bits."""
    g = hub_graph()
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    widths = (0,) if schedule == "plain" else (0, 64, 128, 256)
    for kb in widths:
        for fp64 in (False, True):
            # the graph's first jobs at a width run the tuner's trials
            for _ in range(3):
                ctx.exact(G, schedule=schedule, batch_k=kb, delta_fp64=fp64)
            a = ctx.exact(G, schedule=schedule, batch_k=kb, delta_fp64=fp64).copy()
            assert_bc_close(a, ref, fp64)
            b = ctx.exact(G, schedule=schedule, batch_k=kb, delta_fp64=fp64).copy()
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), (schedule, kb, fp64)
    if schedule == "batch_vertex":
        assert ctx.last_stats()["chunk_edges"] == 0
    if schedule in ("batch_warp", "batch_edge"):
        assert ctx.last_stats()["chunk_edges"] == (256 if schedule == "batch_warp" else 128)
    ctx.destroy_graph(G)


def test_tuner_picks_width_and_split_per_graph():
    """The first jobs with enough sources run the width trial (256, 128 and 64
    sources per batch, twice each), the work-split trial and the concurrent
    groups trial on their own batches; every result matches the oracle, later
    jobs keep the choices, and they repeat bit for bit."""
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(13, 16, seed=11)  # exact BC: 8192 sources, automatic width 256
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    with bc.Context(0) as fresh:
        G = fresh.create_graph(g.row_ptr, g.col_idx)
        for _ in range(3):
            assert_bc_close(fresh.exact(G).copy(), ref, False)
        st1 = fresh.last_stats()
        assert st1["batch_sources"] in (64, 128, 256)
        assert st1["batch_groups"] in (1, 2, 4)
        later = [fresh.exact(G).copy() for _ in range(2)]
        st2 = fresh.last_stats()
        for key in ("batch_sources", "batch_groups", "chunk_edges", "grab"):
            assert st2[key] == st1[key], key
        assert (st2["chunk_edges"], st2["grab"]) in ((256, 2), (128, 2), (512, 2), (256, 1), (0, 2))
        for x in later:
            assert_bc_close(x, ref, False)
        assert np.array_equal(later[0].view(np.uint64), later[1].view(np.uint64))
        # FP64 dependencies on the tuned configuration
        assert_bc_close(fresh.exact(G, delta_fp64=True), ref, True)
        fresh.destroy_graph(G)


def test_plain_block_and_grid_forms_agree(ctx):
    """The one-source-per-launch schedule runs a small graph's sources as
    one-block launches on several streams at once, and a single source (or a
    large graph) as one launch over the whole GPU: both forms against the
    oracle, and one-source jobs summed equal the many-source job."""
    g = bcgen.rmat(10, 8, seed=1)  # the one-source-per-launch benchmark graph
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    srcs = bcgen.sample_sources(g.n, 40, seed=2)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    for fp64 in (True, False):
        many = ctx.sources(G, srcs, schedule="plain", delta_fp64=fp64).copy()
        assert_bc_close(many, ref, fp64)
        assert ctx.last_stats()["kernel_kind"] == 1 and ctx.last_stats()["batches"] == len(srcs)
    one = sum(ctx.sources(G, [int(s_)], schedule="plain", delta_fp64=True).copy() for s_ in srcs)
    assert_bc_close(one, ref, True)
    # the captured launches are replayed for later jobs of the same size: other
    # sources, another graph, the same graph again
    g2 = bcgen.rmat(10, 8, seed=7)
    G2 = ctx.create_graph(g2.row_ptr, g2.col_idx)
    for gg, GG, seed in ((g, G, 5), (g2, G2, 6), (g, G, 2)):
        ss = bcgen.sample_sources(gg.n, 40, seed=seed)
        rr, _ = oracle.bc(gg.n, gg.row_ptr, gg.col_idx, ss)
        assert_bc_close(ctx.sources(GG, ss, schedule="plain", delta_fp64=True), rr, True)
    ctx.destroy_graph(G2)
    full, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    assert_bc_close(ctx.exact(G, schedule="plain", delta_fp64=True), full, True)
    ctx.destroy_graph(G)


@pytest.mark.parametrize("direction", ["pull", "push"])
def test_32_bit_count_rows_match_64_bit(ctx, direction):
    """Path counts stored in 32 bits (the default) give the same depths,
    counts and BC bits as 64-bit storage, pulled or pushed, at every batch
    width; both match the oracle."""
    for g in (bcgen.rmat(11, 16, seed=5), bcgen.ba_directed(2500, 8, 9, seed=3), hub_graph()):
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
        for kb in (64, 128, 256):
            for fp64 in (False, True):
                # one fixed work split, so both runs add in the same order
                a = ctx.exact(G, batch_k=kb, delta_fp64=fp64, direction=direction,
                              count_bits=32, schedule="batch_warp").copy()
                b = ctx.exact(G, batch_k=kb, delta_fp64=fp64, direction=direction,
                              count_bits=64, schedule="batch_warp").copy()
                assert_bc_close(a, ref, fp64)
                assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), (kb, fp64)
        srcs = [0, 3, g.n - 1]
        d, sig, _ = ctx.debug_sources(G, srcs, delta_fp64=True, direction=direction)
        for j, s_ in enumerate(srcs):
            od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, s_)
            np.testing.assert_array_equal(d[j], od)
            np.testing.assert_array_equal(sig[j], osig)
        ctx.destroy_graph(G)


@pytest.mark.parametrize("direction", ["pull", "push"])
def test_counts_beyond_32_bits_promote_the_job(direction):
    """A count of 2^32 or more does not fit the 32-bit rows: the job reruns
    with 64-bit counts (and later jobs on the graph keep them); results and
    counts stay exact, and 2^64 still overflows as the oracle says."""
    import paper_1409_7764_gb300 as bc
    with bc.Context(0) as fresh:
        g = bcgen.layered_chain(40, 3)  # 3^40 (about 1.2e19) paths: beyond 32 bits, within 64
        G = fresh.create_graph(g.row_ptr, g.col_idx)
        ref, ovf = oracle.bc(g.n, g.row_ptr, g.col_idx)
        assert not ovf.any()
        assert_bc_close(fresh.exact(G, delta_fp64=True, direction=direction), ref, True)
        assert_bc_close(fresh.exact(G, delta_fp64=False, direction=direction), ref, False)
        d, sig, _ = fresh.debug_sources(G, [0, 1], delta_fp64=True, direction=direction)
        for j, s_ in enumerate([0, 1]):
            od, osig, _, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, s_)
            np.testing.assert_array_equal(d[j], od)
            np.testing.assert_array_equal(sig[j], osig)
        assert int(sig[0].max()) > 2 ** 32
        fresh.destroy_graph(G)
        bad = bcgen.layered_chain(41, 3)  # 3^41 > 2^64: overflow, flagged like the oracle
        G = fresh.create_graph(bad.row_ptr, bad.col_idx)
        with pytest.raises(bc.BCError) as ei:
            fresh.sources(G, [0, 2], direction=direction)
        assert ei.value.status == bc.BC_ERR_SIGMA_OVERFLOW
        _, ovf = oracle.bc(bad.n, bad.row_ptr, bad.col_idx, [0, 2])
        assert ei.value.stats["overflow_sources"] == int(np.count_nonzero(ovf))
        fresh.destroy_graph(G)


@pytest.mark.parametrize("groups", [2, 4])
def test_concurrent_batch_groups(groups, monkeypatch):
    """A job's batches after its trials running several at a time, each group
    of thread blocks on its own workspace and BC partial vector: exact and
    sampled BC against the oracle, both precisions, both count widths, and a
    repeated job gives the same bits."""
    import paper_1409_7764_gb300 as bc
    monkeypatch.setenv("BC_GROUPS", str(groups))
    g = bcgen.rmat(12, 16, seed=4)
    srcs = bcgen.sample_sources(g.n, 1500, seed=8)
    ref_all, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    ref_s, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    with bc.Context(0) as fresh:
        G = fresh.create_graph(g.row_ptr, g.col_idx)
        for _ in range(2):  # the width and split trials
            fresh.exact(G)
        for fp64 in (False, True):
            for bits in (0, 64):
                a = fresh.exact(G, delta_fp64=fp64, count_bits=bits).copy()
                assert_bc_close(a, ref_all, fp64)
                assert fresh.last_stats()["batch_groups"] == groups
                b = fresh.exact(G, delta_fp64=fp64, count_bits=bits).copy()
                assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
                assert_bc_close(fresh.sources(G, srcs, delta_fp64=fp64, count_bits=bits,
                                              batch_k=64), ref_s, fp64)
        fresh.destroy_graph(G)


@pytest.mark.parametrize("kb,active", [(256, 306), (256, 356), (128, 168), (256, 456)])
def test_last_batch_narrow_and_sources_without_out_edges(ctx, kb, active):
    """Sources without out-edges are ordered last and not launched (their
    traversal is the source alone and adds nothing); the last batch of the
    others, when at most half full, runs with fewer mask words in the wide
    batches' layout (64 of 256, 128 of 256, 64 of 128).  BC against the
    oracle in both precisions and count widths, the same bits on a repeat,
    and a list of such sources alone gives zeros without a launch."""
    g = bcgen.rmat(12, 16, seed=6)
    outdeg = np.diff(g.row_ptr)
    act = np.flatnonzero(outdeg > 0).astype(np.int32)
    sinks = np.flatnonzero(outdeg == 0).astype(np.int32)
    rs = np.random.default_rng(active)
    srcs = np.concatenate([rs.choice(act, active, replace=False), sinks[:30]]).astype(np.int32)
    rs.shuffle(srcs)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    for fp64 in (False, True):
        for bits in (0, 64):
            a = ctx.sources(G, srcs, delta_fp64=fp64, batch_k=kb, count_bits=bits).copy()
            assert_bc_close(a, ref, fp64)
            assert ctx.last_stats()["batches"] == -(-active // kb)
            b = ctx.sources(G, srcs, delta_fp64=fp64, batch_k=kb, count_bits=bits).copy()
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    none = ctx.sources(G, np.tile(sinks[:40], 8), batch_k=kb)
    assert not none.any() and ctx.last_stats()["batches"] == 0
    ctx.destroy_graph(G)


def test_512_edge_split_with_unsplit_long_entries(monkeypatch):
    """With 512-edge chunks, entries of 257..512 in+out edges run as single
    unsplit items started with the hubs' chunks (and larger hubs as chunks):
    BC against the oracle in both precisions and count widths, exact and
    sampled, pulled and pushed, and a repeated job gives the same bits."""
    import paper_1409_7764_gb300 as bc
    monkeypatch.setenv("BC_SPLIT", "2")  # the 512-edge candidate of the tuner
    g = bcgen.rmat(12, 16, seed=3)  # 66 vertices with 257..512 edges, 13 above
    deg = np.diff(g.row_ptr) + np.bincount(g.col_idx, minlength=g.n)
    assert ((deg > 256) & (deg <= 512)).sum() > 10 and (deg > 512).sum() > 5
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    srcs = bcgen.sample_sources(g.n, 700, seed=5)
    sref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    with bc.Context(0) as fresh:
        G = fresh.create_graph(g.row_ptr, g.col_idx)
        for fp64 in (False, True):
            for bits in (0, 64):
                for direction in ("pull", "push"):
                    a = fresh.exact(G, delta_fp64=fp64, count_bits=bits, direction=direction,
                                    batch_k=256).copy()
                    assert fresh.last_stats()["chunk_edges"] == 512
                    assert_bc_close(a, ref, fp64)
                    b = fresh.exact(G, delta_fp64=fp64, count_bits=bits, direction=direction,
                                    batch_k=256).copy()
                    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
                    assert_bc_close(fresh.sources(G, srcs, delta_fp64=fp64, count_bits=bits,
                                                  direction=direction, batch_k=128), sref, fp64)
        fresh.destroy_graph(G)


def test_tuning_remembered_when_a_graph_is_created_again():
    """A large graph destroyed and created again in the same context starts
    with the tuning its first copy found: its first job runs no trials (the
    same batches as the tuned copy's jobs) and gives the tuned copy's bits."""
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(17, 16, seed=2)
    assert g.m >= 1 << 20
    srcs = bcgen.sample_sources(g.n, 4096, seed=3)
    keys = ("batch_sources", "mask_words", "chunk_edges", "grab", "batch_groups", "batches")
    with bc.Context(0) as fresh:
        G = fresh.create_graph(g.row_ptr, g.col_idx)
        for _ in range(3):  # the width, split and groups trials
            fresh.sources(G, srcs)
        tuned = fresh.sources(G, srcs).copy()
        st = fresh.last_stats()
        fresh.destroy_graph(G)
        G2 = fresh.create_graph(g.row_ptr, g.col_idx)
        again = fresh.sources(G2, srcs).copy()
        st2 = fresh.last_stats()
        for key in keys:
            assert st2[key] == st[key], key
        assert np.array_equal(again.view(np.uint64), tuned.view(np.uint64))
        ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs[:64])
        assert_bc_close(fresh.sources(G2, srcs[:64]), ref, False)
        fresh.destroy_graph(G2)
