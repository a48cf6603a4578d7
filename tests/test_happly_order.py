"""The order of the beta single excitations in the FP32 H-apply's mixed
alpha-beta groups (Eq. 2), checked on the CPU.

Every order of a column's singles gives the same contributions (the mixed
groups of an alpha single sum over the column's beta singles j -> b), so the
order must be a permutation of the column's singles, for every column.  The
library chooses it so that the eight lanes of one wavefront of 16-byte
shared-memory loads (eight consecutive columns) read the staged table item
of their single and the staged source row of their partner string from
distinct bank groups where it can: counted here, from the definitions of
the two indices, against the natural order.
"""
from collections import defaultdict
from math import comb

import numpy as np
import pytest


@pytest.fixture(scope="module")
def uc():
    from paper_2402_17993_gb300 import build
    build.build()
    import paper_2402_17993_gb300 as uc
    return uc


def _singles(n_orb, s):
    return [(j, b) for j in range(n_orb) if (s >> j) & 1 for b in range(n_orb) if not (s >> b) & 1]


def _wavefronts(n_orb, n_beta, order):
    """16-byte loads per slot and group of eight columns: the largest number
    of distinct table items (sources) in one of the eight bank groups, the
    source counted twice (two chunks)."""
    strs = [s for s in range(1 << n_orb) if bin(s).count("1") == n_beta]
    rank = {s: i for i, s in enumerate(strs)}
    tot = 0
    for q0 in range(0, len(strs), 8):
        cols = range(q0, min(q0 + 8, len(strs)))
        for t in range(order.shape[0]):
            items, srcs = set(), set()
            for c in cols:
                s = strs[c]
                j, b = _singles(n_orb, s)[order[t, c]]
                lo, hi = min(j, b), max(j, b)
                between = ((1 << hi) - 1) & ~((2 << lo) - 1)
                pi = bin(s & between).count("1") & 1
                items.add(j * n_orb + b + n_orb * n_orb * pi)
                srcs.add(rank[s ^ (1 << j) ^ (1 << b)])
            gi, gs = defaultdict(int), defaultdict(int)
            for v in items:
                gi[v % 8] += 1
            for v in srcs:
                gs[v % 8] += 1
            tot += max(gi.values()) + 2 * max(gs.values())
    return tot


@pytest.mark.parametrize("n_orb,n_beta", [(4, 2), (5, 1), (6, 3), (8, 4), (9, 4), (9, 5)])
def test_order_is_a_permutation_per_column(uc, n_orb, n_beta):
    order = uc.happly_mixed_order(n_orb, n_beta)
    ns = n_beta * (n_orb - n_beta)
    assert order.shape == (ns, comb(n_orb, n_beta))
    assert np.array_equal(np.sort(order, axis=0),
                          np.broadcast_to(np.arange(ns)[:, None], order.shape))
    assert np.array_equal(order, uc.happly_mixed_order(n_orb, n_beta))  # deterministic


@pytest.mark.parametrize("n_orb,n_beta", [(6, 3), (8, 4), (9, 5)])
def test_order_cuts_bank_conflicts(uc, n_orb, n_beta):
    order = uc.happly_mixed_order(n_orb, n_beta)
    natural = np.broadcast_to(np.arange(order.shape[0])[:, None], order.shape)
    got, nat = _wavefronts(n_orb, n_beta, order), _wavefronts(n_orb, n_beta, natural)
    floor = 3 * order.shape[0] * ((order.shape[1] + 7) // 8)
    assert floor <= got < nat
    if n_orb == 9:  # the 18-qubit dimer fragments: within 5% of one wavefront per load
        assert got <= 1.05 * floor


def test_order_rejects_bad_sizes(uc):
    with pytest.raises(uc.UCCSDError):
        uc.happly_mixed_order(16, 8)
    with pytest.raises(uc.UCCSDError):
        uc.happly_mixed_order(4, 5)
    assert uc.happly_mixed_order(4, 0).shape == (0, 1)
