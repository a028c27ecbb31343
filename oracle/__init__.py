"""CPU oracle for exact betweenness centrality -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product (the CUDA library and its
Python binding) never imports, links or executes it, and shares no code with
it.

The arithmetic lives in ``brandes.c`` (classical sequential Brandes, exact
uint64 path counts with carry detection, FP64 dependencies, compensated FP64
sums); see that file's header for the definition it follows (paper,
Section I) and the readings taken where the paper is silent.

Pinned by ``tests/test_oracle.py`` against closed forms, an exact rational
brute force built from walk counting, the path-sum invariant and, when
available, NetworkX (the paper's own validator, Section II.A).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brandes.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile brandes.c (plain -O2, no fast-math) into _oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC",
                               "-shared", "-std=c11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_bc.restype = ctypes.c_int
        lib.oracle_bc.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int32, f64p, i32p]
        lib.oracle_single_source.restype = ctypes.c_int32
        lib.oracle_single_source.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p,
                                             u64p, f64p, i32p]
        lib.oracle_canonicalise.restype = ctypes.c_int64
        lib.oracle_canonicalise.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p]
        lib.oracle_canonical_edges.restype = ctypes.c_int64
        lib.oracle_canonical_edges.argtypes = [ctypes.c_int32, i32p, i32p]
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def bc(n: int, row_ptr, col_idx, sources=None):
    """Raw (unnormalised) betweenness over `sources` (all vertices in id
    order when None).  Returns (bc float64[n], overflow int32[k])."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    out = np.zeros(max(n, 1), dtype=np.float64)
    if sources is None:
        k = n
        src_p = None
    else:
        src = _i32(sources)
        k = int(src.shape[0])
        src_p = _ptr(src if k else np.zeros(1, np.int32), ctypes.c_int32)
    ovf = np.zeros(max(k, 1), dtype=np.int32)
    rc = _load().oracle_bc(n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32), src_p, k,
                           _ptr(out, ctypes.c_double), _ptr(ovf, ctypes.c_int32))
    if rc != 0:
        raise ValueError(f"oracle_bc failed ({rc}): invalid graph or source")
    return out[:n].copy(), ovf[:k].copy()


def single_source(n: int, row_ptr, col_idx, s: int):
    """(d int32[n], sigma uint64[n], delta float64[n], overflow bool) for one
    source; unreached vertices have d = -1, sigma = 0, delta = 0."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    d = np.empty(max(n, 1), dtype=np.int32)
    sig = np.empty(max(n, 1), dtype=np.uint64)
    dl = np.empty(max(n, 1), dtype=np.float64)
    ovf = ctypes.c_int32(0)
    rc = _load().oracle_single_source(n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32), s,
                                      _ptr(d, ctypes.c_int32), _ptr(sig, ctypes.c_uint64),
                                      _ptr(dl, ctypes.c_double), ctypes.byref(ovf))
    if rc < 0:
        raise ValueError(f"oracle_single_source failed ({rc})")
    return d[:n].copy(), sig[:n].copy(), dl[:n].copy(), bool(ovf.value)


def canonicalise(n: int, row_ptr, col_idx):
    """The oracle's own canonical CSR: (row_ptr, col_idx)."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    orp = np.empty(n + 1, dtype=np.int32)
    oci = np.empty(max(int(rp[-1]), 1), dtype=np.int32)
    m = _load().oracle_canonicalise(n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                                    _ptr(orp, ctypes.c_int32), _ptr(oci, ctypes.c_int32))
    if m < 0:
        raise ValueError("invalid CSR")
    return orp, oci[:m].copy()


def source_terms(n: int, row_ptr, col_idx, sources) -> np.ndarray:
    """Per-source BC terms x[i, v] = delta_{s_i}(v) for v != s_i and 0 for
    v == s_i (the terms whose sum over sources is BC, paper Section I), one
    row per given source, from the sequential single-source Brandes above."""
    src = _i32(sources)
    x = np.zeros((src.size, n), dtype=np.float64)
    for i, s_ in enumerate(src):
        _, _, dl, _ = single_source(n, row_ptr, col_idx, int(s_))
        x[i] = dl
        x[i, int(s_)] = 0.0
    return x


def sampled_estimate(n: int, row_ptr, col_idx, sources):
    """Estimate of BC from k sources drawn uniformly without replacement from
    the n vertices, with its standard error.  Sampling is cited in the paper
    (Section I) without an estimator; this is the textbook one: with x_s(v)
    the per-source terms above, the sample mean m(v) and the sample variance
    S2(v) = sum_s (x_s(v) - m(v))^2 / (k - 1) (two-pass, from the definition),
        estimate(v) = n * m(v),
        stderr(v)   = n * sqrt((1 - k/n) * S2(v) / k)
    (the finite-population correction (1 - k/n) makes stderr 0 when every
    vertex is a source).  Returns (estimate, stderr); stderr is NaN for k < 2."""
    x = source_terms(n, row_ptr, col_idx, sources)
    k = x.shape[0]
    m = x.mean(axis=0) if k else np.zeros(n)
    est = n * m
    if k < 2:
        return est, np.full(n, np.nan)
    s2 = ((x - m) ** 2).sum(axis=0) / (k - 1)
    return est, n * np.sqrt((1.0 - k / n) * s2 / k)


def normalise(bc_raw: np.ndarray, n: int) -> np.ndarray:
    """Directed normalisation 1/((n-1)(n-2)) for n > 2 (NetworkX's
    normalized=True convention for DiGraphs); identity otherwise."""
    if n <= 2:
        return bc_raw.copy()
    return bc_raw / float((n - 1) * (n - 2))
