"""The sweeps' entry maps (the sector index of every tile entry, by which a
run reads and writes its tiles in the sector order), checked on the CPU.

For every run of a plan, the map must send the tile entries of all its tiles
one to one onto the sector indices (alpha rank x C(n_orb, n_beta) + beta
rank), and each entry's index must be the one of its determinant, which the
check hook decodes by another route (tile strings deposited into the tile's
qubit positions) and this test ranks by itself.
"""
from math import comb

import numpy as np
import pytest


@pytest.fixture(scope="module")
def uc():
    from paper_2402_17993_gb300 import build
    build.build()
    import paper_2402_17993_gb300 as uc
    return uc


def _sector_index(n_orb, na, nb, det):
    """Alpha orbital i is qubit 2i, beta orbital j qubit 2j + 1."""
    sa = sum(((det >> (2 * i)) & 1) << i for i in range(n_orb))
    sb = sum(((det >> (2 * j + 1)) & 1) << j for j in range(n_orb))
    ra = sum(1 for s in range(sa) if bin(s).count("1") == na)
    rb = sum(1 for s in range(sb) if bin(s).count("1") == nb)
    return ra * comb(n_orb, nb) + rb, bin(sa).count("1"), bin(sb).count("1")


@pytest.mark.parametrize("n_orb,na,nb", [(4, 2, 2), (6, 3, 3), (5, 3, 1), (7, 4, 3)])
@pytest.mark.parametrize("amp_bytes,nvec", [(8, 1), (16, 2)])
def test_entry_maps_are_the_sector_order(uc, n_orb, na, nb, amp_bytes, nvec):
    ijab = uc.build_uccsd_list(n_orb, na, nb)
    rows = uc.plan_entry_map(n_orb, na, nb, ijab, amp_bytes, nvec).astype(np.int64)
    D = comb(n_orb, na) * comb(n_orb, nb)
    runs = np.unique(rows[:, 0])
    assert len(runs) >= 1
    for r in runs:
        sel = rows[rows[:, 0] == r]
        # one to one onto the sector, over all tiles of the run
        assert np.array_equal(np.sort(sel[:, 3]), np.arange(D)), r
        # entries of a tile are 0..n-1 in order
        for t in np.unique(sel[:, 1]):
            e = sel[sel[:, 1] == t][:, 2]
            assert np.array_equal(e, np.arange(len(e)))
    cache = {}
    for det, idx in zip(rows[:, 4].tolist(), rows[:, 3].tolist()):
        if det not in cache:
            cache[det] = _sector_index(n_orb, na, nb, det)
        want, pa, pb = cache[det]
        assert (pa, pb) == (na, nb)
        assert idx == want


def test_entry_map_rejects_bad_input(uc):
    ex = uc.build_uccsd_list(4, 2, 2)
    with pytest.raises(uc.UCCSDError):
        uc.plan_entry_map(4, 2, 2, ex, 12, 1)
    bad = ex.copy()
    bad[0, 2] = 1  # an occupied target orbital
    with pytest.raises(uc.UCCSDError):
        uc.plan_entry_map(4, 2, 2, bad, 8, 1)
