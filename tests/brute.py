"""Exact brute-force betweenness for tiny graphs, independent of Brandes.

Two separate constructions, both in exact rational arithmetic:

* ``bc_by_paths``: enumerate every simple path from every source by DFS,
  keep the shortest ones per (s, t) and count, per interior vertex, the
  fraction of them through it (the definition in the paper's Section I,
  written out literally).  Exponential; n <= 9.
* ``bc_by_walks``: all-pairs distances by Floyd-Warshall, path counts as
  walk counts sigma_st = (A^d(s,t))[s, t] (every walk of length d(s,t) is a
  shortest path), and sigma_st(v) = sigma_sv * sigma_vt exactly when
  d(s,v) + d(v,t) = d(s,t).  Polynomial; n <= ~40.
"""
from fractions import Fraction

import numpy as np

INF = 1 << 60


def adjacency(g):
    a = [[0] * g.n for _ in range(g.n)]
    src, dst = g.edges()
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            a[u][v] = 1
    return a


def floyd_warshall(a):
    n = len(a)
    d = [[0 if i == j else (1 if a[i][j] else INF) for j in range(n)] for i in range(n)]
    for k in range(n):
        dk = d[k]
        for i in range(n):
            dik = d[i][k]
            if dik >= INF:
                continue
            di = d[i]
            for j in range(n):
                if dik + dk[j] < di[j]:
                    di[j] = dik + dk[j]
    return d


def walk_counts(a, d):
    """sigma[s][t] = number of walks of length d(s,t) from s to t."""
    n = len(a)
    sigma = [[0] * n for _ in range(n)]
    power = [[1 if i == j else 0 for j in range(n)] for i in range(n)]  # A^0
    maxd = max([x for row in d for x in row if x < INF] + [0])
    for length in range(0, maxd + 1):
        for s in range(n):
            for t in range(n):
                if d[s][t] == length:
                    sigma[s][t] = power[s][t]
        # power <- power @ A (exact Python ints)
        power = [[sum(power[i][k] * a[k][j] for k in range(n) if power[i][k]) for j in range(n)]
                 for i in range(n)]
    return sigma


def bc_by_walks(g, sources=None):
    a = adjacency(g)
    d = floyd_warshall(a)
    sigma = walk_counts(a, d)
    n = g.n
    srcs = range(n) if sources is None else sources
    bc = [Fraction(0)] * n
    for s in srcs:
        for t in range(n):
            if t == s or d[s][t] >= INF:
                continue
            for v in range(n):
                if v == s or v == t:
                    continue
                if d[s][v] + d[v][t] == d[s][t]:
                    bc[v] += Fraction(sigma[s][v] * sigma[v][t], sigma[s][t])
    return bc, d, sigma


def dependencies_by_walks(g, s):
    """delta_s(v) = sum_t sigma_st(v) / sigma_st, exact."""
    a = adjacency(g)
    d = floyd_warshall(a)
    sigma = walk_counts(a, d)
    n = g.n
    out = [Fraction(0)] * n
    for t in range(n):
        if t == s or d[s][t] >= INF:
            continue
        for v in range(n):
            if v == t:
                continue
            if d[s][v] + d[v][t] == d[s][t]:
                out[v] += Fraction(sigma[s][v] * sigma[v][t], sigma[s][t])
    return out


def bc_by_paths(g):
    a = adjacency(g)
    n = g.n
    nbrs = [[j for j in range(n) if a[i][j]] for i in range(n)]
    bc = [Fraction(0)] * n
    for s in range(n):
        best = {}  # t -> (length, [paths])
        stack = [(s, [s])]
        while stack:
            v, p = stack.pop()
            if v != s:
                L = len(p) - 1
                cur = best.get(v)
                if cur is None or L < cur[0]:
                    best[v] = (L, [p])
                elif L == cur[0]:
                    cur[1].append(p)
            for w in nbrs[v]:
                if w not in p:
                    stack.append((w, p + [w]))
        for t, (_, paths) in best.items():
            cnt = len(paths)
            for p in paths:
                for v in p[1:-1]:
                    bc[v] += Fraction(1, cnt)
    return bc
