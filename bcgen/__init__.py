"""Seeded synthetic inputs for betweenness-centrality runs.

This package only builds inputs: canonical CSR graphs (R-MAT, directed
preferential attachment, closed-form families) and seeded source lists.  It
holds none of the centrality arithmetic, so it can feed both the CPU oracle
and the CUDA library without the two sharing method code.

The input families follow the paper's setting (Section II.C: synthetic
scale-free directed graphs, Barabasi-Albert growth) and the standard R-MAT
recipe (a, b, c, d) = (0.57, 0.19, 0.19, 0.05).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_bcgen.so")
_lib = None

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def build(force: bool = False) -> str:
    """Compile gen.c into _bcgen.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.bcg_splitmix64.restype = ctypes.c_uint64
        lib.bcg_splitmix64.argtypes = [ctypes.c_uint64]
        lib.bcg_rmat_edges.restype = ctypes.c_int64
        lib.bcg_rmat_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_int32, i32p, i32p]
        lib.bcg_ba_edges.restype = ctypes.c_int64
        lib.bcg_ba_edges.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_uint64, i32p, i32p]
        lib.bcg_csr_from_edges.restype = ctypes.c_int64
        lib.bcg_csr_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p]
        lib.bcg_sample_sources.restype = ctypes.c_int32
        lib.bcg_sample_sources.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p]
        lib.bcg_uniform_ints.restype = None
        lib.bcg_uniform_ints.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_uint64, i32p]
        lib.bcg_permutation.restype = None
        lib.bcg_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, i32p]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


@dataclass
class Graph:
    """Directed graph in CSR form: out-neighbours of v are
    col_idx[row_ptr[v]:row_ptr[v+1]]."""
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col_idx: np.ndarray  # int32 [m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col_idx.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self):
        src = np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_ptr))
        return src, self.col_idx


def splitmix64(x: int) -> int:
    return int(_load().bcg_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def csr_from_edges(n: int, src, dst, name: str = "") -> Graph:
    """Canonical CSR (sorted rows, no duplicates, no self-loops)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(max(m, 1), dtype=np.int32)
    got = _load().bcg_csr_from_edges(n, m, _p(src), _p(dst), _p(row_ptr), _p(col))
    if got < 0:
        raise ValueError("edge endpoint out of range")
    return Graph(n, row_ptr, col[:got].copy(), name)


def raw_csr_from_edges(n: int, src, dst, name: str = "") -> Graph:
    """CSR that keeps duplicates, self-loops and input order (for testing
    canonicalisation in the consumers)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int32)
    order = np.argsort(src, kind="stable")
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return Graph(n, row_ptr, dst[order].astype(np.int32), name)


def rmat(scale: int, edge_factor: int, seed: int = 1, abcd=RMAT_ABCD,
         permute: bool = True) -> Graph:
    """Directed R-MAT graph with n = 2^scale, n*edge_factor raw edges,
    self-loops and duplicates removed."""
    n = 1 << scale
    ne = n * edge_factor
    src = np.empty(ne, dtype=np.int32)
    dst = np.empty(ne, dtype=np.int32)
    a, b, c, _ = abcd
    got = _load().bcg_rmat_edges(scale, ne, a, b, c, ctypes.c_uint64(seed), int(permute),
                                 _p(src), _p(dst))
    if got != ne:
        raise ValueError("bad R-MAT arguments")
    return csr_from_edges(n, src, dst, name=f"rmat-s{scale}-ef{edge_factor}-seed{seed}")


def ba_directed(n: int, out_edges: int = 8, m0: int = 9, seed: int = 1) -> Graph:
    """Directed preferential attachment: complete digraph on m0 seed
    vertices, then each new vertex u links u -> t to `out_edges` distinct
    existing vertices t drawn with probability proportional to t's total
    degree.  Vertex ids are arrival order (not relabelled)."""
    total = m0 * (m0 - 1) + out_edges * (n - m0)
    src = np.empty(total, dtype=np.int32)
    dst = np.empty(total, dtype=np.int32)
    got = _load().bcg_ba_edges(n, m0, out_edges, ctypes.c_uint64(seed), _p(src), _p(dst))
    if got != total:
        raise ValueError("bad preferential-attachment arguments")
    return csr_from_edges(n, src, dst, name=f"ba-n{n}-out{out_edges}-seed{seed}")


def ba_undirected(n: int, beta: int, seed: int = 1) -> Graph:
    """Undirected preferential attachment with every edge stored in both
    directions (the paper's synthetic workload, Section III: m is about
    2*beta*n directed edges, edge density d = m/n from 2 to 60).  Seed: a
    clique on beta+1 vertices; then each new vertex joins beta distinct
    existing vertices drawn with probability proportional to their degree.
    Built from the directed generator (whose total degree is the undirected
    degree) by adding the reverse of every edge."""
    if beta < 1 or n < beta + 1:
        raise ValueError("need beta >= 1 and n >= beta + 1")
    g = ba_directed(n, beta, beta + 1, seed)
    a, b = g.edges()
    return csr_from_edges(n, np.concatenate([a, b]), np.concatenate([b, a]),
                          name=f"ba-undirected-n{n}-beta{beta}-seed{seed}")


def sample_sources(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct sources uniform over [0, n) (seeded partial Fisher-Yates)."""
    out = np.empty(max(k, 1), dtype=np.int32)
    if _load().bcg_sample_sources(n, k, ctypes.c_uint64(seed), _p(out)) != k:
        raise ValueError("k must be in [0, n]")
    return out[:k].copy()


def uniform_ints(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.int32)
    _load().bcg_uniform_ints(count, lo, hi, ctypes.c_uint64(seed), _p(out))
    return out[:count].copy()


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.int32)
    _load().bcg_permutation(n, ctypes.c_uint64(seed), _p(out))
    return out[:n].copy()


def small_rmat_specs(count: int, master_seed: int = 1, scale_lo: int = 6, scale_hi: int = 12,
                     ef_lo: int = 4, ef_hi: int = 16):
    """(scale, edge_factor, seed) for a batch of small R-MAT graphs: scale and
    edge factor integer-uniform from two splitmix64 streams, graph i seeded by
    splitmix64(master_seed ^ i)."""
    scales = uniform_ints(count, scale_lo, scale_hi, splitmix64(master_seed ^ 0x5CA1E))
    efs = uniform_ints(count, ef_lo, ef_hi, splitmix64(master_seed ^ 0xEF))
    return [(int(scales[i]), int(efs[i]), splitmix64(master_seed ^ i)) for i in range(count)]


# ---- closed-form families ------------------------------------------------

def path(n: int, bidirected: bool = False) -> Graph:
    s = np.arange(n - 1)
    src, dst = s, s + 1
    if bidirected:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    return csr_from_edges(n, src, dst, name=f"path{'-bi' if bidirected else ''}-{n}")


def cycle(n: int) -> Graph:
    s = np.arange(n)
    return csr_from_edges(n, s, (s + 1) % n, name=f"cycle-{n}")


def star(n: int, kind: str = "bi") -> Graph:
    """Centre 0 with leaves 1..n-1; kind 'bi' (both directions), 'out' or 'in'."""
    leaves = np.arange(1, n)
    zero = np.zeros(n - 1, dtype=np.int64)
    if kind == "out":
        src, dst = zero, leaves
    elif kind == "in":
        src, dst = leaves, zero
    else:
        src, dst = np.concatenate([zero, leaves]), np.concatenate([leaves, zero])
    return csr_from_edges(n, src, dst, name=f"star-{kind}-{n}")


def complete(n: int) -> Graph:
    u, v = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mask = u != v
    return csr_from_edges(n, u[mask], v[mask], name=f"complete-{n}")


def grid(rows: int, cols: int) -> Graph:
    """Directed rows x cols grid with right and down edges; vertex (i, j) has
    id i*cols + j."""
    src, dst = [], []
    for i in range(rows):
        for j in range(cols):
            v = i * cols + j
            if j + 1 < cols:
                src.append(v); dst.append(v + 1)
            if i + 1 < rows:
                src.append(v); dst.append(v + cols)
    return csr_from_edges(rows * cols, src, dst, name=f"grid-{rows}x{cols}")


def layered_chain(q: int, width: int = 2) -> Graph:
    """Source 0, then q stages; each stage fans out to `width` middle vertices
    which all join into the stage's sink.  The sink of stage i is the source
    of stage i+1.  Shortest-path count at the last sink is width^q."""
    src, dst = [], []
    cur = 0
    nxt = 1
    for _ in range(q):
        mids = list(range(nxt, nxt + width))
        sink = nxt + width
        for mid in mids:
            src += [cur, mid]
            dst += [mid, sink]
        cur = sink
        nxt = sink + 1
    return csr_from_edges(nxt, src, dst, name=f"chain-{width}^{q}")


def random_digraph(n: int, p: float, seed: int) -> Graph:
    """Erdos-Renyi directed graph G(n, p), seeded (for tiny brute-force cases)."""
    rs = np.random.default_rng(seed)
    adj = rs.random((n, n)) < p
    np.fill_diagonal(adj, False)
    u, v = np.nonzero(adj)
    return csr_from_edges(n, u, v, name=f"gnp-{n}-{p}-{seed}")
