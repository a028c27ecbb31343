"""The seeded input generators: structural properties of the undirected
preferential-attachment graphs the paper measures on (Section III: every
undirected edge stored as two directed ones, m about 2*beta*n), checked
without the oracle."""
from collections import deque

import numpy as np
import pytest

import bcgen


def _adjacency_sets(g):
    return [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]


@pytest.mark.parametrize("n,beta", [(500, 1), (2000, 3), (3000, 30)])
def test_ba_undirected_structure(n, beta):
    g = bcgen.ba_undirected(n, beta, seed=5)
    adj = _adjacency_sets(g)
    # symmetric, no self-loops, canonical rows
    for v in range(g.n):
        assert v not in adj[v]
        row = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert (np.diff(row) > 0).all()
        for x in adj[v]:
            assert v in adj[x]
    # a clique on beta+1 seed vertices, then beta new undirected edges per vertex
    assert g.m == 2 * (beta * (beta + 1) // 2 + beta * (n - beta - 1))
    for v in range(beta + 1):
        assert set(range(beta + 1)) - {v} <= adj[v]
    deg = g.out_degree()
    assert deg.min() >= beta
    # vertex v > beta joined exactly beta older vertices
    for v in range(beta + 1, n):
        assert sum(1 for x in adj[v] if x < v) == beta
    # connected (every arrival joins the existing component)
    seen = np.zeros(n, dtype=bool)
    seen[0] = True
    q = deque([0])
    while q:
        v = q.popleft()
        for x in adj[v]:
            if not seen[x]:
                seen[x] = True
                q.append(x)
    assert seen.all()
    # preferential attachment: early vertices collect far more edges
    assert deg[: n // 100 + 1].mean() > 3 * deg[n // 2:].mean()


def test_ba_undirected_seeded():
    a = bcgen.ba_undirected(1000, 4, seed=3)
    b = bcgen.ba_undirected(1000, 4, seed=3)
    c = bcgen.ba_undirected(1000, 4, seed=4)
    assert np.array_equal(a.col_idx, b.col_idx) and np.array_equal(a.row_ptr, b.row_ptr)
    assert not np.array_equal(a.col_idx, c.col_idx)
    with pytest.raises(ValueError):
        bcgen.ba_undirected(3, 3)
