"""bc_sources_noalloc: the entry point for callers that cannot allocate.

Callers that may not call cudaMalloc (a fixed memory budget reserved at
start-up, an allocator that owns all device memory, a callback that must not
stall) pass the graph and the output as device memory they own; the library
keeps its working state in one fixed array and allocates nothing.  This test
calls that entry point through the C ABI twice in a row and checks each
result against bc_sources on the same graph and sources, within the parity
tolerances (1e-12 relative for FP64 dependencies, 1e-4 for FP32).  It lives in
a file collected last and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import bcgen

pytestmark = pytest.mark.gpu


def in_csr(g):
    src, dst = g.edges()
    order = np.lexsort((src, dst))
    in_idx = src[order].astype(np.int32)
    in_ptr = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(in_ptr, dst.astype(np.int64) + 1, 1)
    return np.cumsum(in_ptr).astype(np.int32), in_idx


def close(got, ref, tol):
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero])
    rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
    assert rel.max() <= tol, f"max rel err {rel.max():.3e}"


def test_noalloc_matches_bc_sources_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    import paper_1409_7764_gb300 as bc
    from paper_1409_7764_gb300 import capi
    lib = bc.load()
    g = bcgen.rmat(12, 8, seed=5)  # n = 4096, hubs with hundreds of edges
    ip, ii = in_csr(g)
    dev = torch.device("cuda", 0)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    ci_d = torch.from_numpy(g.col_idx).to(dev)
    ip_d = torch.from_numpy(ip).to(dev)
    ii_d = torch.from_numpy(ii).to(dev)
    out = torch.empty(g.n, dtype=torch.float64, device=dev)
    srcs = np.concatenate([bcgen.sample_sources(g.n, 130, seed=3), [7, 7]]).astype(np.int32)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def call(fp64, sources=srcs, n=g.n):
        return lib.bc_sources_noalloc(rp_d.data_ptr(), ci_d.data_ptr(), ip_d.data_ptr(),
                                      ii_d.data_ptr(), n, g.m, sources.ctypes.data,
                                      len(sources), int(fp64), out.data_ptr(), stream)

    with bc.Context(0) as ctx:
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        for fp64, tol in [(True, 1e-12), (False, 1e-4)]:
            ref = ctx.sources(G, srcs, delta_fp64=fp64)
            for _ in range(2):
                out.fill_(-1.0)
                assert call(fp64) == bc.BC_OK
                torch.cuda.synchronize()
                close(out.cpu().numpy(), ref, tol)
        ctx.destroy_graph(G)

    # sizes beyond the fixed array and bad sources are refused before any work
    assert call(True, n=capi.BC_NOALLOC_MAX_N + 1) == bc.BC_ERR_ARG
    assert call(True, sources=np.array([g.n], dtype=np.int32)) == bc.BC_ERR_ARG
