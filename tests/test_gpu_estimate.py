"""Sampled-source estimator on the GPU (bc_sources_estimate, bc_sources_adaptive)
against the oracle's estimator (tests/test_oracle_estimator.py pins it).

Bars: estimate within the BC parity tolerance (1e-12 FP64 / 1e-4 FP32
dependencies); standard error within 1e-9 (FP64) / 1e-3 (FP32) relative, since
it is the square root of a variance formed from the same terms (their
rounding enters once, halved by the root); exact zeros stay zero.
"""
import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu

EST_TOL = {True: 1e-12, False: 1e-4}
ERR_TOL = {True: 1e-9, False: 1e-3}


@pytest.fixture(scope="module")
def ctx():
    import paper_1409_7764_gb300 as bc
    c = bc.Context(0)
    yield c
    c.close()


def close(got, ref, tol):
    got, ref = np.asarray(got), np.asarray(ref)
    zero = ref == 0
    assert np.all(np.abs(got[zero]) <= tol * (np.abs(ref).max() + 1e-300))
    if (~zero).any():
        rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
        assert rel.max() <= tol, f"max rel err {rel.max():.3e}"


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("k,kb", [(300, 0), (700, 256), (129, 64)])
def test_estimate_matches_oracle(ctx, fp64, k, kb):
    g = bcgen.rmat(11, 8, seed=4)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    src = bcgen.sample_sources(g.n, k, seed=k)
    est, err = ctx.estimate(G, src, delta_fp64=fp64, batch_k=kb)
    oest, oerr = oracle.sampled_estimate(g.n, g.row_ptr, g.col_idx, src)
    close(est, oest, EST_TOL[fp64])
    close(err, oerr, ERR_TOL[fp64])
    # normalised outputs scale both by 1/((n-1)(n-2))
    nest, nerr = ctx.estimate(G, src, delta_fp64=fp64, batch_k=kb, normalize=True)
    f = 1.0 / ((g.n - 1) * (g.n - 2))
    np.testing.assert_allclose(nest, est * f, rtol=1e-15)
    np.testing.assert_allclose(nerr, err * f, rtol=1e-15)
    ctx.destroy_graph(G)


def test_all_sources_exact_with_zero_error(ctx):
    g = bcgen.rmat(9, 8, seed=2)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    est, err = ctx.estimate(G, np.arange(g.n), delta_fp64=True)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    close(est, ref, 1e-12)
    assert np.all(err == 0.0)
    _, err1 = ctx.estimate(G, [3], delta_fp64=True)
    assert np.isnan(err1).all()
    ctx.destroy_graph(G)


def test_adaptive_sampling_stops_at_the_first_round_meeting_the_target(ctx):
    g = bcgen.rmat(11, 16, seed=6)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    order = bcgen.sample_sources(g.n, g.n, seed=3)  # a seeded permutation
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    min_est = float(np.quantile(ref, 0.99))
    rel, rnd = 0.15, 128
    est, err, used = ctx.adaptive(G, order, rel, round=rnd, min_est=min_est, delta_fp64=True)
    assert 2 <= used <= g.n and (used % rnd == 0 or used == g.n)
    top = est >= min_est
    assert np.all(err[top] <= rel * est[top])
    # the result is the estimate over the sources used ...
    e2, r2 = ctx.estimate(G, order[:used], delta_fp64=True)
    close(est, e2, 1e-12)
    close(err, r2, 1e-9)
    oest, oerr = oracle.sampled_estimate(g.n, g.row_ptr, g.col_idx, order[:used])
    close(est, oest, 1e-12)
    close(err, oerr, 1e-9)
    # ... and one round fewer had not met the target
    if used > rnd:
        e3, r3 = ctx.estimate(G, order[:used - rnd], delta_fp64=True)
        t3 = e3 >= min_est
        assert np.any(r3[t3] > rel * e3[t3])
    # a cap on the sources is honoured
    _, _, capped = ctx.adaptive(G, order, 1e-6, round=100, max_k=250, min_est=min_est)
    assert capped == 250
    ctx.destroy_graph(G)


def test_estimator_argument_errors(ctx):
    import paper_1409_7764_gb300 as bc
    g = bcgen.rmat(6, 4, seed=1)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    for call in (lambda: ctx.estimate(G, [g.n]),
                 lambda: ctx.adaptive(G, np.arange(g.n), 0.0),
                 lambda: ctx.adaptive(G, np.arange(g.n), 0.1, round=0)):
        with pytest.raises(bc.BCError) as ei:
            call()
        assert ei.value.status == bc.BC_ERR_ARG
    ctx.destroy_graph(G)
