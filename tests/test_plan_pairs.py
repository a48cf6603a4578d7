"""The excitation sweeps' precomputed pair lists, checked on the CPU
against the oracle's generators (Eq. 4).

For every excitation of a list, the lists of the sweep plan must hold each
pair of determinants that G_k connects inside the electron sector exactly
once, over all tiles and runs, in an order and with a sign such that the
sweep's rotation
    first' = c first - sign s second,   second' = c second + sign s first
is exp(theta G_k) on that pair.  With G_k|x> = s_k |x'> for the occupied
side x (Eq. 4's tau_k|x> up to the sign), that means (first, second, sign)
is (x, x', s_k) or (x', x, -s_k).  Within a factor's list every group of
16 pairs (8 for 16-byte amplitudes), the lanes of one shared-memory
wavefront, uses distinct residues of its first entries and distinct
residues of its second entries (no bank conflicts).  Forward (one vector)
and adjoint (two vectors) plans, FP32 and FP64 amplitudes.
"""
import functools

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def uc():
    from paper_2402_17993_gb300 import build
    build.build()
    import paper_2402_17993_gb300 as uc
    return uc


@functools.lru_cache(maxsize=None)
def _basis(n, na, nb):
    return oracle.sector_basis(n, na, nb)


def _oracle_pairs(n, na, nb, row):
    """(occupied side x, partner x', s) with G|x> = s|x'> over the sector."""
    basis = _basis(n, na, nb)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[basis] = np.arange(1, len(basis) + 1)
    g = oracle.apply_generator(n, row, psi).real
    ys = np.nonzero(g)[0]
    vals = g[ys]
    xs = basis[np.rint(np.abs(vals)).astype(np.int64) - 1]
    occ = sum(1 << int(q) for q in (row[0], row[1]) if q >= 0)
    vir = sum(1 << int(q) for q in (row[2], row[3]) if q >= 0)
    side = ((xs & occ) == occ) & ((xs & vir) == 0)
    return xs[side], ys[side], np.sign(vals[side]).astype(np.int64)


@pytest.mark.parametrize("n_orb,na,nb", [(4, 2, 2), (6, 3, 3), (5, 3, 1), (9, 5, 5)])
@pytest.mark.parametrize("amp_bytes,nvec", [(8, 1), (8, 2), (16, 1), (16, 2)])
def test_pair_lists_equal_the_generators(uc, n_orb, na, nb, amp_bytes, nvec):
    n = 2 * n_orb
    ijab = uc.build_uccsd_list(n_orb, na, nb)
    rows = uc.plan_pairs(n_orb, na, nb, ijab, amp_bytes, nvec).astype(np.int64)
    real = rows[:, 1] >= 0
    assert np.all((rows[:, 1] < 0) == (rows[:, 2] < 0))
    assert set(np.unique(rows[:, 3])) <= {-1, 1}
    pr = rows[real]
    pr = pr[np.argsort(pr[:, 0], kind="stable")]
    bounds = np.searchsorted(pr[:, 0], np.arange(len(ijab) + 1))
    for k in range(len(ijab)):
        r = pr[bounds[k]:bounds[k + 1]]
        x, xp, s = _oracle_pairs(n, na, nb, ijab[k])
        assert len(r) == len(x), k
        # oriented as the oracle's pair, with the oracle's sign, or swapped
        # with the opposite sign; every oracle pair exactly once
        okey = (x << 32) | xp
        order = np.argsort(okey)
        okey, os_ = okey[order], s[order]
        fwd = (r[:, 1] << 32) | r[:, 2]
        rev = (r[:, 2] << 32) | r[:, 1]
        i_f = np.clip(np.searchsorted(okey, fwd), 0, len(okey) - 1)
        i_r = np.clip(np.searchsorted(okey, rev), 0, len(okey) - 1)
        is_f = okey[i_f] == fwd
        is_r = okey[i_r] == rev
        assert np.all(is_f ^ is_r), k
        idx = np.where(is_f, i_f, i_r)
        expect = np.where(is_f, os_[idx], -os_[idx])
        assert np.array_equal(r[:, 3], expect), k
        assert len(np.unique(idx)) == len(okey), k
    # bank groups: each factor's list (it restarts at index 0) in groups of G
    G = 16 if amp_bytes == 8 else 8
    starts = np.nonzero(rows[:, 6] == 0)[0].tolist() + [len(rows)]
    for a, b in zip(starts[:-1], starts[1:]):
        lst = rows[a:b]
        assert len(lst) % G == 0
        for g0 in range(0, len(lst), G):
            grp = lst[g0:g0 + G]
            assert len(set((grp[:, 4] % G).tolist())) == G
            assert len(set((grp[:, 5] % G).tolist())) == G


def test_plan_pairs_rejects_bad_input(uc):
    ex = uc.build_uccsd_list(4, 2, 2)
    with pytest.raises(uc.UCCSDError):
        uc.plan_pairs(4, 2, 2, ex, 12, 1)
    with pytest.raises(uc.UCCSDError):
        uc.plan_pairs(4, 2, 2, ex, 8, 3)
    bad = ex.copy()
    bad[0, 2] = 1  # an occupied target orbital
    with pytest.raises(uc.UCCSDError):
        uc.plan_pairs(4, 2, 2, bad, 8, 1)
