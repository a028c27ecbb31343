"""Pins for the CPU oracle (no GPU).

The oracle is the reference the CUDA path is compared with, so it is itself
checked against things other than itself: closed forms, two exact rational
brute forces built without Brandes' recurrence, the path-length sum
invariant, per-source invariants and NetworkX (the validator the paper used,
Section II.A).
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import bcgen
import oracle
from tests import brute


def obc(g, sources=None):
    return oracle.bc(g.n, g.row_ptr, g.col_idx, sources)


# ---- closed forms ----------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 10, 37])
def test_directed_path(n):
    g = bcgen.path(n)
    bc, ovf = obc(g)
    i = np.arange(n)
    np.testing.assert_array_equal(bc, i * (n - 1 - i))
    assert not ovf.any()


@pytest.mark.parametrize("n", [2, 5, 16])
def test_bidirected_path(n):
    bc, _ = obc(bcgen.path(n, bidirected=True))
    i = np.arange(n)
    np.testing.assert_array_equal(bc, 2 * i * (n - 1 - i))


@pytest.mark.parametrize("n", [3, 4, 9, 20])
def test_directed_cycle(n):
    bc, _ = obc(bcgen.cycle(n))
    np.testing.assert_array_equal(bc, np.full(n, (n - 1) * (n - 2) / 2))


@pytest.mark.parametrize("n", [3, 6, 50])
def test_star(n):
    bc, _ = obc(bcgen.star(n, "bi"))
    expect = np.zeros(n)
    expect[0] = (n - 1) * (n - 2)
    np.testing.assert_array_equal(bc, expect)
    # one-directional stars have no interior vertex at all; the out-star
    # catches a source wrongly credited with its own dependency
    np.testing.assert_array_equal(obc(bcgen.star(n, "out"))[0], np.zeros(n))
    np.testing.assert_array_equal(obc(bcgen.star(n, "in"))[0], np.zeros(n))


@pytest.mark.parametrize("n", [2, 5, 12])
def test_complete_digraph(n):
    g = bcgen.complete(n)
    bc, _ = obc(g)
    np.testing.assert_array_equal(bc, np.zeros(n))
    d, sig, dl, ovf = oracle.single_source(g.n, g.row_ptr, g.col_idx, 0)
    assert d[0] == 0 and (d[1:] == 1).all()
    assert (sig == 1).all()
    assert not ovf


def test_grid_counts_are_binomials():
    rows, cols = 7, 9
    g = bcgen.grid(rows, cols)
    d, sig, _, ovf = oracle.single_source(g.n, g.row_ptr, g.col_idx, 0)
    for i in range(rows):
        for j in range(cols):
            assert d[i * cols + j] == i + j
            assert int(sig[i * cols + j]) == comb(i + j, i)
    assert not ovf


@pytest.mark.parametrize("width,q", [(2, 10), (2, 63), (3, 40)])
def test_layered_chain_counts_exact(width, q):
    g = bcgen.layered_chain(q, width)
    d, sig, _, ovf = oracle.single_source(g.n, g.row_ptr, g.col_idx, 0)
    assert int(sig[g.n - 1]) == width ** q
    assert d[g.n - 1] == 2 * q
    assert not ovf


@pytest.mark.parametrize("width,q", [(2, 64), (3, 41)])
def test_layered_chain_overflow_flagged(width, q):
    # width^q >= 2^64: the count no longer fits and the source is flagged
    g = bcgen.layered_chain(q, width)
    _, sig, _, ovf = oracle.single_source(g.n, g.row_ptr, g.col_idx, 0)
    assert ovf
    _, flags = obc(g, [0, 1])
    assert flags.tolist() == [1, 0]


# ---- exact brute force -------------------------------------------------------

def _tiny_graphs():
    out = []
    for seed in range(6):
        out.append(bcgen.random_digraph(7, 0.35, seed))
    out.append(bcgen.random_digraph(9, 0.25, 11))
    out.append(bcgen.random_digraph(8, 0.6, 12))
    return out


@pytest.mark.parametrize("g", _tiny_graphs(), ids=lambda g: g.name)
def test_matches_path_enumeration(g):
    exact = brute.bc_by_paths(g)
    bc, _ = obc(g)
    for v in range(g.n):
        if exact[v] == 0:
            assert bc[v] == 0.0
        else:
            assert abs(Fraction(bc[v]) - exact[v]) <= exact[v] * Fraction(1, 10**15)


def _small_graphs():
    out = [bcgen.random_digraph(n, p, seed)
           for (n, p, seed) in [(12, 0.2, 1), (16, 0.15, 2), (24, 0.1, 3), (30, 0.08, 4),
                                (20, 0.3, 5)]]
    out.append(bcgen.rmat(5, 4, seed=3))
    out.append(bcgen.ba_directed(30, out_edges=3, m0=4, seed=2))
    out.append(bcgen.ba_undirected(28, beta=2, seed=4))
    return out


@pytest.mark.parametrize("g", _small_graphs(), ids=lambda g: g.name)
def test_matches_walk_counting(g):
    exact, _, _ = brute.bc_by_walks(g)
    bc, _ = obc(g)
    for v in range(g.n):
        if exact[v] == 0:
            assert bc[v] == 0.0
        else:
            assert abs(Fraction(bc[v]) - exact[v]) <= exact[v] * Fraction(1, 10**14)


def test_dependencies_and_counts_match_walk_counting():
    g = bcgen.random_digraph(18, 0.18, 7)
    a = brute.adjacency(g)
    dist = brute.floyd_warshall(a)
    sigma = brute.walk_counts(a, dist)
    for s in range(g.n):
        d, sig, dl, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, s)
        exact = brute.dependencies_by_walks(g, s)
        for v in range(g.n):
            if dist[s][v] >= brute.INF:
                assert d[v] == -1 and sig[v] == 0 and dl[v] == 0.0
                continue
            assert d[v] == dist[s][v]
            assert int(sig[v]) == sigma[s][v]
            assert abs(Fraction(dl[v]) - exact[v]) <= (exact[v] + 1) * Fraction(1, 10**14)


def test_sampled_sources_and_duplicates():
    g = bcgen.random_digraph(20, 0.15, 9)
    srcs = [3, 7, 7, 15]
    exact, _, _ = brute.bc_by_walks(g, sources=srcs)
    bc, flags = obc(g, srcs)
    assert flags.tolist() == [0, 0, 0, 0]
    for v in range(g.n):
        assert abs(Fraction(bc[v]) - exact[v]) <= (exact[v] + 1) * Fraction(1, 10**14)
    # a source list is a plain sum of per-source results
    parts = sum(obc(g, [s])[0] for s in srcs)
    np.testing.assert_allclose(bc, parts, rtol=1e-14, atol=0)


# ---- invariants --------------------------------------------------------------

def _all_pairs_hops(g):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    a = csr_matrix((np.ones(g.m), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    return shortest_path(a, method="D", directed=True, unweighted=True)


@pytest.mark.parametrize("g", [bcgen.rmat(8, 8, seed=1), bcgen.rmat(9, 4, seed=2),
                               bcgen.ba_directed(400, 4, 5, seed=3),
                               bcgen.ba_undirected(400, 3, seed=3)], ids=lambda g: g.name)
def test_sum_invariant(g):
    """sum_v BC[v] = sum over reachable ordered pairs s != t of (d(s,t) - 1):
    each shortest s-t path has d(s,t) - 1 interior vertices."""
    dist = _all_pairs_hops(g)
    fin = np.isfinite(dist) & (dist > 0)
    rhs = int((dist[fin] - 1).sum())
    bc, _ = obc(g)
    assert abs(bc.sum() - rhs) <= 1e-12 * max(rhs, 1)


def test_per_source_invariants():
    g = bcgen.rmat(9, 8, seed=5)
    dist = _all_pairs_hops(g)
    src, dst = g.edges()
    for s in [0, 1, 17, 200, 511]:
        d, sig, dl, _ = oracle.single_source(g.n, g.row_ptr, g.col_idx, s)
        reach = np.isfinite(dist[s])
        np.testing.assert_array_equal(d[reach], dist[s][reach].astype(np.int32))
        assert (d[~reach] == -1).all()
        nr = int(reach.sum())
        # delta_s(s) counts every reachable target once
        assert abs(dl[s] - (nr - 1)) <= 1e-9 * nr
        # the dependencies of s sum to the interior-vertex count of its paths
        rhs = float((dist[s][reach & (dist[s] > 0)] - 1).sum())
        lhs = dl.sum() - dl[s]
        assert abs(lhs - rhs) <= 1e-10 * max(rhs, 1)
        # sigma[w] is the sum of sigma over its shortest-path predecessors
        on_dag = (d[src] >= 0) & (d[dst] == d[src] + 1)
        acc = np.zeros(g.n, dtype=object)
        for u, w in zip(src[on_dag], dst[on_dag]):
            acc[w] += int(sig[u])
        for w in range(g.n):
            if d[w] > 0:
                assert acc[w] == int(sig[w])


# ---- library cross-check -----------------------------------------------------

def test_networkx_cross_check():
    nx = pytest.importorskip("networkx")
    for g in [bcgen.rmat(7, 6, seed=4), bcgen.ba_directed(150, 3, 4, seed=1),
              bcgen.random_digraph(60, 0.05, 8)]:
        G = nx.DiGraph()
        G.add_nodes_from(range(g.n))
        s, d = g.edges()
        G.add_edges_from(zip(s.tolist(), d.tolist()))
        ref = nx.betweenness_centrality(G, normalized=False)
        bc, _ = obc(g)
        np.testing.assert_allclose(bc, [ref[v] for v in range(g.n)], rtol=1e-11, atol=1e-9)
        refn = nx.betweenness_centrality(G, normalized=True)
        np.testing.assert_allclose(oracle.normalise(bc, g.n), [refn[v] for v in range(g.n)],
                                   rtol=1e-11, atol=1e-12)


def test_networkx_undirected_cross_check():
    """On a graph with every edge in both directions (the paper's undirected
    preferential-attachment inputs), the sum over ordered pairs counts each
    unordered pair twice: BC = 2 x NetworkX's undirected betweenness."""
    nx = pytest.importorskip("networkx")
    for g in [bcgen.ba_undirected(200, 1, seed=1), bcgen.ba_undirected(150, 4, seed=2)]:
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        s, d = g.edges()
        G.add_edges_from(zip(s.tolist(), d.tolist()))
        ref = nx.betweenness_centrality(G, normalized=False)
        bc, _ = obc(g)
        np.testing.assert_allclose(bc, [2 * ref[v] for v in range(g.n)], rtol=1e-11, atol=1e-9)


# ---- input handling ------------------------------------------------------------

def test_canonicalisation_removes_duplicates_and_loops():
    rs = np.random.default_rng(0)
    n = 40
    src = rs.integers(0, n, 300)
    dst = rs.integers(0, n, 300)
    src = np.concatenate([src, src[:50], np.arange(10)])  # duplicates + self-loops
    dst = np.concatenate([dst, dst[:50], np.arange(10)])
    raw = bcgen.raw_csr_from_edges(n, src, dst)
    canon = bcgen.csr_from_edges(n, src, dst)
    rp, ci = oracle.canonicalise(n, raw.row_ptr, raw.col_idx)
    np.testing.assert_array_equal(rp, canon.row_ptr)
    np.testing.assert_array_equal(ci, canon.col_idx)
    np.testing.assert_array_equal(obc(raw)[0], obc(canon)[0])


def test_rejects_malformed_csr():
    with pytest.raises(ValueError):
        oracle.bc(3, [0, 2, 1, 2], [1, 2])  # non-monotone row_ptr
    with pytest.raises(ValueError):
        oracle.bc(3, [0, 1, 1, 2], [1, 5])  # column out of range
    with pytest.raises(ValueError):
        oracle.bc(3, [1, 1, 1, 2], [1, 2])  # row_ptr[0] != 0
    with pytest.raises(ValueError):
        oracle.bc(3, [0, 1, 1, 1], [1], sources=[3])  # bad source


def test_empty_and_edgeless():
    bc, _ = oracle.bc(0, [0], [])
    assert bc.shape == (0,)
    bc, _ = oracle.bc(5, [0] * 6, [])
    np.testing.assert_array_equal(bc, np.zeros(5))
