"""Helper of the FMO two-body tests (no test of its own)."""
import numpy as np


def dimer_theta(ex_i, th_i, ex_j, th_j, ex_d, nocc, nvir):
    """Amplitudes of a dimer's excitation list from its monomers' (spin
    orbitals remapped from [occ, virt] of a monomer to [occ I, occ J,
    virt I, virt J] of the dimer); cross-fragment rows get zero."""
    def remap(q, frag):
        if q < 0:
            return q
        p, s = q >> 1, q & 1
        new = (frag * nocc + p) if p < nocc else (2 * nocc + frag * nvir + (p - nocc))
        return 2 * new + s
    table = {}
    for frag, (ex, th) in enumerate(((ex_i, th_i), (ex_j, th_j))):
        for row, t in zip(ex.tolist(), th):
            table[tuple(remap(q, frag) for q in row)] = t
    return np.array([table.get(tuple(r), 0.0) for r in ex_d.tolist()])
