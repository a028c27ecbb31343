"""Serving: jobs submitted while others run are admitted and overlap on the
device; each result is the same alone and in the mix (within the parity
tolerance) and matches the oracle; oversized jobs are refused."""
import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu


def close(got, ref, tol):
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero])
    if (~zero).any():
        rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
        assert rel.max() <= tol, f"max rel err {rel.max():.3e}"


def test_alone_versus_mix():
    import paper_1409_7764_gb300 as bc
    from paper_1409_7764_gb300.serving import Request, poisson_arrivals, run_open_loop, summarize
    gs = [bcgen.rmat(9, 16, seed=1), bcgen.rmat(11, 8, seed=2), bcgen.ba_directed(3000, 4, 5, 3),
          bcgen.rmat(13, 16, seed=4)]
    with bc.Context(0) as ctx:
        hs = [ctx.create_graph(g.row_ptr, g.col_idx) for g in gs]
        reqs = [Request(hs[0], None, dict(delta_fp64=True)),
                Request(hs[1], None, dict(delta_fp64=False)),
                Request(hs[2], bcgen.sample_sources(3000, 200, seed=5), dict(delta_fp64=True)),
                Request(hs[3], bcgen.sample_sources(hs[3].n, 512, seed=6),
                        dict(delta_fp64=False, scale_sampled=True))]
        tols = [1e-12, 1e-4, 1e-12, 1e-4]
        alone = []
        for r in reqs:
            job = ctx.submit(r.graph, r.sources, **r.opts)
            st, out, _ = ctx.wait(job, r.graph.n)
            assert st == 0
            alone.append(out.copy())
        # the mix: three rounds of all four, arriving within a few milliseconds
        mix = reqs * 3
        results = {}
        recs = run_open_loop(ctx, mix, poisson_arrivals(len(mix), 2000.0, seed=9),
                             results=results)
        s = summarize(recs)
        assert s["errors"] == 0 and s["requests"] == len(mix)
        for i, r in enumerate(mix):
            close(results[i], alone[i % 4], tols[i % 4])
        # and against the oracle
        for i, (g, r) in enumerate(zip(gs, reqs)):
            ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, r.sources)
            if r.opts.get("scale_sampled"):
                ref = ref * g.n / len(r.sources)
            close(alone[i], ref, tols[i])
        for h in hs:
            ctx.destroy_graph(h)


def test_poll_semantics_and_admission():
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(8, 8, seed=3)
    with bc.Context(0) as ctx:
        G = ctx.create_graph(g.row_ptr, g.col_idx)
        job = ctx.submit(G, None, delta_fp64=True)
        st, out, stats = ctx.wait(job, g.n)
        assert st == 0 and stats["sources"] == g.n
        with pytest.raises(bc.BCError) as ei:
            ctx.poll(job, g.n)  # consumed
        assert ei.value.status == bc.BC_ERR_NOT_FOUND
        # a graph with a job in flight cannot be destroyed
        job = ctx.submit(G, None)
        try:
            ctx.destroy_graph(G)
            destroyed = True
        except bc.BCError as e:
            destroyed = False
            assert e.status == bc.BC_ERR_ARG
        ctx.wait(job, g.n)
        if not destroyed:
            ctx.destroy_graph(G)
    # a budget too small for the job's state: refused at submission
    with bc.Context(0, hbm_budget_bytes=8 << 20) as small:
        big = bcgen.rmat(14, 8, seed=1)
        G = small.create_graph(big.row_ptr, big.col_idx)
        with pytest.raises(bc.BCError) as ei:
            small.submit(G, None)
        assert ei.value.status == bc.BC_ERR_ADMISSION
