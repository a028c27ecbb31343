"""The oracle's pins must be strong enough to catch plausible mistakes.

Each case compiles a copy of the oracle source with one planted mistake (a
dropped term, swapped operands, a wrong comparison, a skipped vertex, the
source credited with its own dependency, a wrong initial count) and checks
that at least one pin rejects it.  Everything runs on the CPU.
"""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import bcgen
import oracle
from tests import brute

SRC = os.path.join(os.path.dirname(oracle.__file__), "brandes.c")

MUTATIONS = {
    "dropped_one": ("(1.0 + w->delta[x])", "(w->delta[x])"),
    "swapped_ratio": ("(double)w->sigma[v] / (double)w->sigma[x]",
                      "(double)w->sigma[x] / (double)w->sigma[v]"),
    "source_credited": ("if (v == s) continue;", ""),
    "wrong_dag_test": ("if (w->d[x] == w->d[v] + 1) {", "if (w->d[x] <= w->d[v] + 1) {"),
    "skipped_last": ("for (int32_t i = tail - 1; i >= 0; --i)",
                     "for (int32_t i = tail - 2; i >= 0; --i)"),
    "sigma_init": ("w->sigma[s] = 1;", "w->sigma[s] = 2;"),
    "no_dedupe": ("if (i == 0 || tmp[i] != tmp[i - 1]) g->adj[out++] = tmp[i];",
                  "g->adj[out++] = tmp[i];"),
    "no_carry_check": ("if (after < before) {", "if (0) {"),
}


def _pins_pass() -> bool:
    """A compact subset of the oracle's pins; False as soon as one fails."""
    try:
        for n in (5, 12):
            bc, _ = oracle.bc(*_csr(bcgen.path(n)))
            i = np.arange(n)
            if not np.array_equal(bc, i * (n - 1 - i)):
                return False
        bc, _ = oracle.bc(*_csr(bcgen.star(9, "out")))
        if bc.any():
            return False
        g = bcgen.grid(5, 6)
        _, sig, _, _ = oracle.single_source(*_csr(g), 0)
        from math import comb
        if any(int(sig[i * 6 + j]) != comb(i + j, i) for i in range(5) for j in range(6)):
            return False
        g = bcgen.layered_chain(64, 2)
        _, _, _, ovf = oracle.single_source(*_csr(g), 0)
        if not ovf:
            return False
        for g in [bcgen.random_digraph(14, 0.2, 1), bcgen.random_digraph(12, 0.3, 2)]:
            exact, _, _ = brute.bc_by_walks(g)
            bc, _ = oracle.bc(*_csr(g))
            for v in range(g.n):
                if abs(Fraction(bc[v]) - exact[v]) > (exact[v] + 1) * Fraction(1, 10**13):
                    return False
        # diamond 0 -> {1, 2} -> 3 with the edge 0 -> 1 doubled: as a simple
        # graph, 1 and 2 each carry half of the single 0 -> 3 pair
        raw = bcgen.raw_csr_from_edges(4, [0, 0, 0, 1, 2], [1, 1, 2, 3, 3])
        bc, _ = oracle.bc(*_csr(raw))
        if not np.array_equal(bc, [0, 0.5, 0.5, 0]):
            return False
    except Exception:
        return False
    return True


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


def test_unmutated_oracle_passes_pins():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "brandes_mut.c"
    mutated.write_text(text.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", str(so),
                           str(mutated)])
    real = oracle._load()
    lib = ctypes.CDLL(str(so))
    for fn in ("oracle_bc", "oracle_single_source", "oracle_canonicalise",
               "oracle_canonical_edges"):
        getattr(lib, fn).restype = getattr(real, fn).restype
        getattr(lib, fn).argtypes = getattr(real, fn).argtypes
    monkeypatch.setattr(oracle, "_lib", lib)
    assert not _pins_pass(), f"planted mistake '{name}' was not caught by any pin"
