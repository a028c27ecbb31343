"""Pins of the oracle's sampled-source estimator (CPU only).

The estimator of BC from k sources sampled uniformly without replacement is
n times the sample mean of the per-source terms, with standard error
n * sqrt((1 - k/n) * S2 / k), S2 the sample variance (k - 1 denominator).
Sampling theory fixes two facts that involve no estimator code: averaged over
all C(n, k) source subsets, the estimate equals the exact BC (unbiasedness),
and the mean of stderr^2 over all subsets equals the actual variance of the
estimate over the subsets.  Both are checked by enumerating every subset of a
small graph, and plausible mistakes (no finite-population correction, a k
denominator, the source's own dependency counted) are shown to fail them.
"""
import itertools

import numpy as np
import pytest

import bcgen
import oracle


def _exact(g):
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx)
    return ref


def _graphs():
    return [bcgen.random_digraph(9, 0.3, 5), bcgen.rmat(3, 4, seed=2),
            bcgen.ba_directed(9, 2, 3, seed=4)]


def _subset_moments(g, k, est_fn):
    ests, errs2 = [], []
    for sub in itertools.combinations(range(g.n), k):
        e, se = est_fn(g.n, g.row_ptr, g.col_idx, np.array(sub, dtype=np.int32))
        ests.append(e)
        errs2.append(se ** 2)
    ests, errs2 = np.array(ests), np.array(errs2)
    return ests.mean(axis=0), ests.var(axis=0), errs2.mean(axis=0)


def _pins_hold(est_fn, g, k):
    mean, var, mean_err2 = _subset_moments(g, k, est_fn)
    scale = np.abs(_exact(g)).max() + 1.0
    return (np.allclose(mean, _exact(g), rtol=1e-12, atol=1e-12 * scale) and
            np.allclose(mean_err2, var, rtol=1e-9, atol=1e-9 * scale ** 2))


@pytest.mark.parametrize("gi", range(3))
@pytest.mark.parametrize("k", [2, 4])
def test_unbiased_and_variance_matches_all_subsets(gi, k):
    g = _graphs()[gi]
    assert _pins_hold(oracle.sampled_estimate, g, k)


def test_all_sources_give_exact_bc_and_zero_error():
    g = bcgen.rmat(7, 6, seed=1)
    est, se = oracle.sampled_estimate(g.n, g.row_ptr, g.col_idx, np.arange(g.n))
    ref = _exact(g)
    np.testing.assert_allclose(est, ref, rtol=1e-12, atol=1e-12)
    assert np.all(se == 0.0)


def test_terms_sum_to_the_other_oracle_path():
    g = bcgen.rmat(6, 8, seed=3)
    src = bcgen.sample_sources(g.n, 20, seed=1)
    x = oracle.source_terms(g.n, g.row_ptr, g.col_idx, src)
    ref, _ = oracle.bc(g.n, g.row_ptr, g.col_idx, src)
    np.testing.assert_allclose(x.sum(axis=0), ref, rtol=1e-12, atol=1e-12)


def test_single_source_has_no_error_estimate():
    g = bcgen.path(6)
    _, se = oracle.sampled_estimate(g.n, g.row_ptr, g.col_idx, [2])
    assert np.isnan(se).all()


def _mutant(kind):
    def est(n, rp, ci, src):
        x = oracle.source_terms(n, rp, ci, src)
        k = x.shape[0]
        if kind == "source_credited":
            for i, s_ in enumerate(src):
                _, _, dl, _ = oracle.single_source(n, rp, ci, int(s_))
                x[i, int(s_)] = dl[int(s_)]
        m = x.mean(axis=0)
        denom = k if kind == "k_denominator" else k - 1
        s2 = ((x - m) ** 2).sum(axis=0) / denom
        fpc = 1.0 if kind == "no_fpc" else 1.0 - k / n
        return n * m, n * np.sqrt(fpc * s2 / k)
    return est


@pytest.mark.parametrize("kind", ["no_fpc", "k_denominator", "source_credited"])
def test_pins_reject_planted_mistakes(kind):
    g = _graphs()[0]
    assert not _pins_hold(_mutant(kind), g, 3)
