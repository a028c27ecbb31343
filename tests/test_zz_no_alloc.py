"""bc_sources_noalloc: the entry point for callers that cannot allocate.

Callers that may not call cudaMalloc (a fixed memory budget reserved at
start-up, an allocator that owns all device memory, a callback that must not
stall) pass the graph and the output as device memory they own; the library
keeps its working state in one fixed array and allocates nothing.  These
tests call that entry point through the C ABI, twice in a row on the same
inputs, and check every result element by element against the CPU oracle
over the same sources (1e-12 relative with FP64 dependencies, 1e-4 with
FP32, exact zeros exact), then against bc_sources as well.  They also check
that a call leaves the device's free memory unchanged, the size limit at
both ends, an overflowing path count and an empty source list.  The file is
collected last and passes both alone and after the other tests.
"""
import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu

TOL = {True: 1e-12, False: 1e-4}


def in_csr(g):
    src, dst = g.edges()
    order = np.lexsort((src, dst))
    in_idx = src[order].astype(np.int32)
    in_ptr = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(in_ptr, dst.astype(np.int64) + 1, 1)
    return np.cumsum(in_ptr).astype(np.int32), in_idx


def close(got, ref, tol):
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero]), "exact zeros differ"
    if (~zero).any():
        rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
        assert rel.max() <= tol, f"max rel err {rel.max():.3e}"


class Caller:
    """The graph in device memory the caller owns, and the raw C call."""

    def __init__(self, g):
        import torch
        import paper_1409_7764_gb300 as bc
        self.torch, self.lib, self.g = torch, bc.load(), g
        ip, ii = in_csr(g)
        dev = torch.device("cuda", 0)
        self.rp = torch.from_numpy(g.row_ptr).to(dev)
        self.ci = torch.from_numpy(g.col_idx if g.m else np.zeros(1, np.int32)).to(dev)
        self.ip = torch.from_numpy(ip).to(dev)
        self.ii = torch.from_numpy(ii if g.m else np.zeros(1, np.int32)).to(dev)
        self.out = torch.empty(max(g.n, 1), dtype=torch.float64, device=dev)
        self.stream = torch.cuda.current_stream(dev).cuda_stream

    def __call__(self, sources, fp64, n=None):
        sources = np.ascontiguousarray(sources, dtype=np.int32)
        self.out.fill_(-1.0)
        rc = self.lib.bc_sources_noalloc(
            self.rp.data_ptr(), self.ci.data_ptr(), self.ip.data_ptr(), self.ii.data_ptr(),
            self.g.n if n is None else n, self.g.m, sources.ctypes.data, len(sources), int(fp64),
            self.out.data_ptr(), self.stream)
        self.torch.cuda.synchronize()
        return rc

    def result(self):
        return self.out.cpu().numpy()[:self.g.n]


def test_noalloc_matches_the_oracle_on_consecutive_calls():
    pytest.importorskip("torch")
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(12, 8, seed=5)  # n = 4096, hubs with hundreds of edges
    sink = int(np.flatnonzero(np.diff(g.row_ptr) == 0)[0])  # a source with no out-edges
    srcs = np.concatenate([bcgen.sample_sources(g.n, 130, seed=3), [7, 7, sink]]).astype(np.int32)
    ref, ovf = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    assert not ovf.any()
    call = Caller(g)
    with bc.Context(0) as ctx:
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        for fp64 in (True, False):
            lib_ref = ctx.sources(G, srcs, delta_fp64=fp64)
            for _ in range(2):
                assert call(srcs, fp64) == bc.BC_OK
                close(call.result(), ref, TOL[fp64])
                close(call.result(), lib_ref, TOL[fp64])
        ctx.destroy_graph(G)
    # a source with no out-edges alone contributes nothing anywhere
    assert call([sink], True) == bc.BC_OK
    assert not call.result().any()


def test_noalloc_allocates_nothing():
    torch = pytest.importorskip("torch")
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(11, 8, seed=2)
    srcs = bcgen.sample_sources(g.n, 100, seed=4)
    call = Caller(g)
    assert call(srcs, False) == bc.BC_OK  # loads the kernels, resolves the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for fp64 in (False, True):
        assert call(srcs, fp64) == bc.BC_OK
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    close(call.result(), ref, TOL[True])


def test_noalloc_at_the_size_limit_and_edge_cases():
    pytest.importorskip("torch")
    import paper_1409_7764_gb300 as bc
    from paper_1409_7764_gb300 import capi
    g = bcgen.rmat(13, 8, seed=9)  # n = 8192 = BC_NOALLOC_MAX_N: the array is full
    assert g.n == capi.BC_NOALLOC_MAX_N
    srcs = bcgen.sample_sources(g.n, 96, seed=6)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, srcs)
    call = Caller(g)
    for _ in range(2):
        assert call(srcs, False) == bc.BC_OK
        close(call.result(), ref, TOL[False])
    # no sources: the output is all zeros
    assert call(np.zeros(0, np.int32), True) == bc.BC_OK
    assert not call.result().any()
    # sizes beyond the fixed array and bad sources are refused before any work
    assert call(srcs, True, n=capi.BC_NOALLOC_MAX_N + 1) == bc.BC_ERR_ARG
    assert call([g.n], True) == bc.BC_ERR_ARG
    assert call([-1], True) == bc.BC_ERR_ARG


def test_noalloc_flags_overflowing_path_counts():
    pytest.importorskip("torch")
    import paper_1409_7764_gb300 as bc
    bad = bcgen.layered_chain(64, 2)  # 2^64 shortest paths from vertex 0 to the last
    call = Caller(bad)
    assert call([0, 1], True) == bc.BC_ERR_SIGMA_OVERFLOW
    ok = bcgen.layered_chain(63, 2)  # 2^63 paths: exact in 64 bits
    call = Caller(ok)
    ref, ovf = oracle.bc(ok.n, ok.row_ptr, ok.col_idx, [0, 1])
    assert not ovf.any()
    assert call([0, 1], True) == bc.BC_OK
    close(call.result(), ref, TOL[True])
