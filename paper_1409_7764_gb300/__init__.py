"""GB300-native exact betweenness centrality (Brandes) -- Python binding.

A thin layer over the C ABI of ``libbc_gb300.so`` (declared in
``include/bc_gb300.h``): it marshals arguments and nothing else.  Every step
of the computation runs in the library's CUDA kernels; there is no CPU
fallback, and loading fails loudly when the library is missing.

Betweenness of v (paper, Section I): the sum over ordered pairs s != v != t of
the fraction of shortest s->t paths through v, on unweighted directed graphs
given as int32 CSR.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import capi
from .capi import (BC_ERR_ADMISSION, BC_ERR_ARG, BC_ERR_CUDA, BC_ERR_GRAPH, BC_ERR_INTERNAL,
                   BC_ERR_NOT_FOUND, BC_ERR_OOM, BC_ERR_SIGMA_OVERFLOW, BC_ERR_TIMEOUT, BC_OK,
                   BC_PENDING, BC_SCHED_AUTO, BC_SCHED_BATCH, BC_SCHED_PLAIN, bc_opts, bc_stats)

__all__ = [
    "BCError", "Context", "Graph", "make_opts", "bc_opts", "bc_stats", "load", "BC_OK",
    "BC_PENDING", "BC_ERR_ARG", "BC_ERR_GRAPH", "BC_ERR_OOM", "BC_ERR_CUDA", "BC_ERR_TIMEOUT",
    "BC_ERR_SIGMA_OVERFLOW", "BC_ERR_NOT_FOUND", "BC_ERR_ADMISSION", "BC_ERR_INTERNAL",
    "BC_SCHED_AUTO", "BC_SCHED_PLAIN", "BC_SCHED_BATCH",
]

_SCHED = {"auto": BC_SCHED_AUTO, "plain": BC_SCHED_PLAIN, "batch": BC_SCHED_BATCH,
          "batch_queue": capi.BC_SCHED_BATCH_QUEUE, "batch_vertex": capi.BC_SCHED_BATCH_VERTEX,
          "batch_warp": capi.BC_SCHED_BATCH_WARP, "batch_edge": capi.BC_SCHED_BATCH_EDGE}


_DIRECTION = {"auto": 0, "pull": 1, "push": 2}


def load():
    """The loaded ctypes library (raises RuntimeError if unavailable)."""
    return capi.load()


class BCError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = capi.load().bc_status_str(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")
        self.bc = None
        self.stats = None


def _check(rc: int, what: str):
    if rc < 0:
        raise BCError(rc, what)
    return rc


def make_opts(delta_fp64: bool = False, batch_k: int = 0, schedule="auto",
              normalize: bool = False, scale_sampled: bool = False,
              out_device: bool = False, keep_source_order: bool = False,
              direction="auto", count_bits: int = 0) -> bc_opts:
    o = bc_opts()
    o.delta_fp64 = int(bool(delta_fp64))
    o.batch_k = int(batch_k)
    o.schedule = _SCHED[schedule] if isinstance(schedule, str) else int(schedule)
    o.normalize = int(bool(normalize))
    o.scale_sampled = int(bool(scale_sampled))
    o.out_device = int(bool(out_device))
    o.source_order = int(bool(keep_source_order))
    o.direction = _DIRECTION[direction] if isinstance(direction, str) else int(direction)
    o.count_bits = int(count_bits)
    return o


@dataclass
class Graph:
    handle: int
    n: int
    m: int


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _out_buffer(out, n):
    """(pointer, out_device flag, holder) for an output vector of n doubles:
    a torch CUDA float64 tensor is written in place on the device, otherwise a
    host numpy array is returned."""
    if out is not None and hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
        if out.numel() != n or str(out.dtype) != "torch.float64" or not out.is_contiguous():
            raise ValueError("device output must be a contiguous float64 tensor of n elements")
        return out.data_ptr(), 1, out
    arr = out if out is not None else np.empty(max(n, 1), dtype=np.float64)
    if arr.dtype != np.float64 or not arr.flags.c_contiguous or arr.size < n:
        raise ValueError("host output must be a contiguous float64 array of n elements")
    return arr.ctypes.data, 0, arr


class Context:
    """One library context on one GPU (bc_init / bc_shutdown)."""

    def __init__(self, device: int = 0, stream=None, hbm_budget_bytes: int = 0):
        self._lib = capi.load()
        h = ctypes.c_void_p()
        _check(self._lib.bc_init(device, _stream_handle(stream), hbm_budget_bytes,
                                 ctypes.byref(h)), "bc_init")
        self._h = h
        self.device = device

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.bc_shutdown(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- graphs -----------------------------------------------------------------
    def create_graph(self, row_ptr, col_idx, n: int | None = None) -> Graph:
        rp, ci = _i32(row_ptr), _i32(col_idx)
        n = int(rp.shape[0] - 1) if n is None else int(n)
        m = int(ci.shape[0])
        g, me = ctypes.c_int64(), ctypes.c_int64()
        ci_ptr = ci.ctypes.data if m else None
        _check(self._lib.bc_create_graph(self._h, rp.ctypes.data, ci_ptr, n, m, ctypes.byref(g),
                                         ctypes.byref(me)), "bc_create_graph")
        return Graph(g.value, n, me.value)

    def create_graphs(self, graphs) -> list:
        """Uploads many graphs with one call; graphs is a sequence of
        (row_ptr, col_idx) pairs (host arrays).  All or nothing."""
        arrs = [(_i32(rp), _i32(ci)) for rp, ci in graphs]
        count = len(arrs)
        if count == 0:
            return []
        rps = (ctypes.c_void_p * count)(*[rp.ctypes.data for rp, _ in arrs])
        cis = (ctypes.c_void_p * count)(*[ci.ctypes.data if ci.size else None for _, ci in arrs])
        ns = np.array([rp.shape[0] - 1 for rp, _ in arrs], dtype=np.int32)
        ms = np.array([ci.shape[0] for _, ci in arrs], dtype=np.int64)
        out = np.empty(count, dtype=np.int64)
        meff = np.empty(count, dtype=np.int64)
        _check(self._lib.bc_create_graphs(self._h, count, rps, cis, ns.ctypes.data, ms.ctypes.data,
                                          out.ctypes.data, meff.ctypes.data), "bc_create_graphs")
        return [Graph(int(h), int(n), int(me)) for h, n, me in zip(out, ns, meff)]

    def destroy_graph(self, g: Graph):
        _check(self._lib.bc_destroy_graph(self._h, g.handle), "bc_destroy_graph")

    # -- synchronous calls ----------------------------------------------------------
    def _finish(self, rc, arr, what):
        if rc == BC_ERR_SIGMA_OVERFLOW:
            err = BCError(rc, what)
            err.bc = arr
            err.stats = self.last_stats()
            raise err
        _check(rc, what)
        return arr

    def exact(self, g: Graph, out=None, **opts):
        ptr, dev, holder = _out_buffer(out, g.n)
        o = make_opts(out_device=dev, **opts)
        rc = self._lib.bc_exact(self._h, g.handle, ctypes.byref(o), ptr)
        res = holder if dev else holder[:g.n]
        return self._finish(rc, res, "bc_exact")

    def sources(self, g: Graph, src, out=None, **opts):
        s = _i32(src)
        ptr, dev, holder = _out_buffer(out, g.n)
        o = make_opts(out_device=dev, **opts)
        rc = self._lib.bc_sources(self._h, g.handle, s.ctypes.data if s.size else None,
                                  int(s.size), ctypes.byref(o), ptr)
        res = holder if dev else holder[:g.n]
        return self._finish(rc, res, "bc_sources")

    def last_overflow_sources(self) -> np.ndarray:
        """Sources whose path count reached 2^64 in the last synchronous call."""
        cnt = ctypes.c_int32(0)
        _check(self._lib.bc_last_overflow_sources(self._h, None, 0, ctypes.byref(cnt)),
               "bc_last_overflow_sources")
        out = np.empty(max(cnt.value, 1), dtype=np.int32)
        _check(self._lib.bc_last_overflow_sources(self._h, out.ctypes.data, cnt.value,
                                                  ctypes.byref(cnt)), "bc_last_overflow_sources")
        return out[:cnt.value].copy()

    def estimate(self, g: Graph, src, out=None, err_out=None, **opts):
        """(estimate, standard error) of BC from the sources `src`, taken as a
        uniform sample without replacement (bc_sources_estimate)."""
        s = _i32(src)
        ptr, dev, holder = _out_buffer(out, g.n)
        eptr, edev, eholder = _out_buffer(err_out, g.n)
        if dev != edev:
            raise ValueError("estimate and error outputs must both be host or both device")
        o = make_opts(out_device=dev, **opts)
        rc = self._lib.bc_sources_estimate(self._h, g.handle, s.ctypes.data if s.size else None,
                                           int(s.size), ctypes.byref(o), ptr, eptr)
        res = (holder, eholder) if dev else (holder[:g.n], eholder[:g.n])
        return self._finish(rc, res, "bc_sources_estimate")

    def adaptive(self, g: Graph, order, rel_err: float, round: int = 1024, max_k=None,
                 min_est: float = 0.0, **opts):
        """(estimate, standard error, sources used): sources taken from
        `order` in rounds until every vertex with estimate >= min_est has a
        relative standard error <= rel_err (bc_sources_adaptive)."""
        s = _i32(order)
        mk = int(s.size if max_k is None else max_k)
        est = np.empty(max(g.n, 1), dtype=np.float64)
        err = np.empty(max(g.n, 1), dtype=np.float64)
        used = ctypes.c_int32(0)
        o = make_opts(**opts)
        rc = self._lib.bc_sources_adaptive(self._h, g.handle, s.ctypes.data if s.size else None,
                                           mk, int(round), float(rel_err), float(min_est),
                                           ctypes.byref(o), est.ctypes.data, err.ctypes.data,
                                           ctypes.byref(used))
        res = (est[:g.n], err[:g.n], int(used.value))
        return self._finish(rc, res, "bc_sources_adaptive")

    def exact_many(self, graphs, out=None, **opts):
        """BC of the graphs in one vector of sum(n) doubles, graph i at offset
        sum_{j<i} n_j.  With `out` a torch CUDA float64 tensor of that length
        the vector is written there on the device and `out` is returned;
        otherwise a list of per-graph host arrays (views of one vector)."""
        hs = np.array([g.handle for g in graphs], dtype=np.int64)
        total = sum(g.n for g in graphs)
        ptr, dev, holder = _out_buffer(out, total)
        o = make_opts(out_device=dev, **opts)
        rc = self._lib.bc_exact_many(self._h, hs.ctypes.data if hs.size else None, len(graphs),
                                     ctypes.byref(o), ptr)
        _check(rc, "bc_exact_many")
        if dev:
            return holder
        res, off = [], 0
        for g in graphs:
            res.append(holder[off:off + g.n])
            off += g.n
        return res

    def last_stats(self) -> dict:
        st = bc_stats()
        _check(self._lib.bc_last_stats(self._h, ctypes.byref(st)), "bc_last_stats")
        return st.as_dict()

    # -- jobs ---------------------------------------------------------------------
    def submit(self, g: Graph, src=None, **opts) -> int:
        o = make_opts(**opts)
        job = ctypes.c_int64()
        if src is None:
            rc = self._lib.bc_submit(self._h, g.handle, None, 0, ctypes.byref(o), ctypes.byref(job))
        else:
            s = _i32(src)
            rc = self._lib.bc_submit(self._h, g.handle, s.ctypes.data if s.size else None,
                                     int(s.size), ctypes.byref(o), ctypes.byref(job))
        _check(rc, "bc_submit")
        return job.value

    def poll(self, job: int, n: int):
        """(status, bc or None, stats dict or None); status BC_PENDING while
        running."""
        out = np.empty(max(n, 1), dtype=np.float64)
        st = bc_stats()
        rc = self._lib.bc_poll(self._h, job, out.ctypes.data, ctypes.byref(st))
        if rc == BC_PENDING:
            return rc, None, None
        if rc in (BC_ERR_NOT_FOUND, BC_ERR_ARG):
            _check(rc, "bc_poll")
        return rc, out[:n], st.as_dict()

    def wait(self, job: int, n: int, timeout_ms: int = -1):
        out = np.empty(max(n, 1), dtype=np.float64)
        st = bc_stats()
        rc = self._lib.bc_wait(self._h, job, timeout_ms, out.ctypes.data, ctypes.byref(st))
        if rc in (BC_ERR_NOT_FOUND, BC_ERR_ARG, BC_ERR_TIMEOUT):
            _check(rc, "bc_wait")
        return rc, out[:n], st.as_dict()

    # -- debug ----------------------------------------------------------------------
    def debug_sources(self, g: Graph, src, **opts):
        """(d int32[k][n], sigma uint64[k][n], delta float64[k][n])."""
        s = _i32(src)
        k = int(s.size)
        d = np.empty((k, g.n), dtype=np.int32)
        sig = np.empty((k, g.n), dtype=np.uint64)
        dl = np.empty((k, g.n), dtype=np.float64)
        o = make_opts(**opts)
        rc = self._lib.bc_debug_sources(self._h, g.handle, s.ctypes.data if k else None, k,
                                        ctypes.byref(o), d.ctypes.data, sig.ctypes.data,
                                        dl.ctypes.data)
        if rc not in (BC_OK, BC_ERR_SIGMA_OVERFLOW):
            _check(rc, "bc_debug_sources")
        return d, sig, dl

    def debug_graph(self, g: Graph):
        """(row_ptr, col_idx, in_ptr, in_idx) as the library holds the graph."""
        rp = np.empty(g.n + 1, dtype=np.int32)
        ci = np.empty(max(g.m, 1), dtype=np.int32)
        ip = np.empty(g.n + 1, dtype=np.int32)
        ii = np.empty(max(g.m, 1), dtype=np.int32)
        _check(self._lib.bc_debug_graph(self._h, g.handle, rp.ctypes.data, ci.ctypes.data,
                                        ip.ctypes.data, ii.ctypes.data), "bc_debug_graph")
        return rp, ci[:g.m], ip, ii[:g.m]

    def debug_source(self, g: Graph, s: int):
        d = np.empty(g.n, dtype=np.int32)
        sig = np.empty(g.n, dtype=np.uint64)
        dl = np.empty(g.n, dtype=np.float64)
        rc = self._lib.bc_debug_source(self._h, g.handle, int(s), d.ctypes.data, sig.ctypes.data,
                                       dl.ctypes.data)
        if rc not in (BC_OK, BC_ERR_SIGMA_OVERFLOW):
            _check(rc, "bc_debug_source")
        return d, sig, dl, rc == BC_ERR_SIGMA_OVERFLOW

    def inject_barrier_skip(self, block: int, timeout_ms: int):
        _check(self._lib.bc_debug_inject_barrier_skip(self._h, block, timeout_ms),
               "bc_debug_inject_barrier_skip")
