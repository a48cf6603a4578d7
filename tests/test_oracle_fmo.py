"""Pins of the oracle's FMO two-body assembly (Section 2.1, Eq. 1), CPU.

* The embedding: the closed-shell reference energy of the whole supersystem
  splits exactly into the embedded monomer's reference energy plus the
  environment's own reference energy (textbook closed-shell sums).
* Eq. 1 for non-interacting fragments: each dimer energy at the monomers'
  amplitudes (cross-fragment amplitudes zero) is the sum of the monomer
  energies, so the two-body total is the sum of the monomer energies.
* Eq. 1 itself against the sum written the other way round.
* The product's fragment integrals (paper_2402_17993_gb300.serving, its own
  code) equal the oracle's element by element."""
import itertools

import numpy as np
import pytest

import synth
from tests._fmo import dimer_theta


def _hf_energy(h, eri, occ):
    """Textbook closed-shell determinant energy over spatial orbitals occ."""
    e = sum(2.0 * h[i, i] for i in occ)
    for i in occ:
        for j in occ:
            e += 2.0 * eri[i, i, j, j] - eri[i, j, j, i]
    return e


@pytest.mark.parametrize("coupling", [0.0, 0.4])
def test_embedded_reference_energy_splits_exactly(oracle_mod, coupling):
    t = synth.fmo_trimer(31, coupling)
    h, eri, fo, fn = t["h"], t["eri"], t["frag_orbs"], t["frag_nocc"]
    occ_all = [o for f in range(3) for o in fo[f][:fn[f]]]
    e_tot = _hf_energy(h, eri, occ_all)
    for members in [(0,), (1,), (2,), (0, 1), (0, 2), (1, 2)]:
        hp, ep, nocc = oracle_mod.fmo_fragment_integrals(h, eri, fo, fn, members)
        n = hp.shape[0]
        ex = oracle_mod.excitations(n, nocc, nocc)
        e_frag = oracle_mod.energy_grad(n, hp, ep, 0.0, nocc, nocc, ex, np.zeros(len(ex)),
                                        grad=False)[0]
        env = [o for f in range(3) if f not in members for o in fo[f][:fn[f]]]
        assert abs(e_frag + _hf_energy(h, eri, env) - e_tot) < 1e-10


def test_non_interacting_fragments_are_additive(oracle_mod):
    t = synth.fmo_trimer(32, 0.0)
    h, eri, fo, fn = t["h"], t["eri"], t["frag_orbs"], t["frag_nocc"]
    mono, thetas, exs = {}, {}, {}
    for i in range(3):
        hp, ep, nocc = oracle_mod.fmo_fragment_integrals(h, eri, fo, fn, (i,))
        exs[i] = oracle_mod.excitations(hp.shape[0], nocc, nocc)
        thetas[i] = synth.theta_normal(len(exs[i]), 0.1, 50 + i)
        mono[i] = oracle_mod.energy_grad(hp.shape[0], hp, ep, 0.0, nocc, nocc, exs[i],
                                         thetas[i], grad=False)[0]
    dim = {}
    for i, j in itertools.combinations(range(3), 2):
        hp, ep, nocc = oracle_mod.fmo_fragment_integrals(h, eri, fo, fn, (i, j))
        ex_d = oracle_mod.excitations(hp.shape[0], nocc, nocc)
        th = dimer_theta(exs[i], thetas[i], exs[j], thetas[j], ex_d, fn[i], len(fo[i]) - fn[i])
        dim[(i, j)] = oracle_mod.energy_grad(hp.shape[0], hp, ep, 0.0, nocc, nocc, ex_d, th,
                                             grad=False)[0]
        assert abs(dim[(i, j)] - mono[i] - mono[j]) < 1e-10
    assert abs(oracle_mod.fmo2_energy(mono, dim, 3) - sum(mono.values())) < 1e-10


def test_fmo2_energy_is_eq1(oracle_mod):
    rng = np.random.default_rng(3)
    for n in (2, 3, 5):
        mono = {i: rng.normal() for i in range(n)}
        dim = {(i, j): rng.normal() for i, j in itertools.combinations(range(n), 2)}
        # Eq. 1 regrouped: sum_{I<J} (E_IJ - E_I - E_J) + sum_I E_I
        alt = sum(dim[k] - mono[k[0]] - mono[k[1]] for k in dim) + sum(mono.values())
        assert abs(oracle_mod.fmo2_energy(mono, dim, n) - alt) < 1e-12


def test_product_fragment_integrals_equal_the_oracle(oracle_mod):
    from paper_2402_17993_gb300 import serving
    t = synth.fmo_trimer(33, 0.3)
    for members in [(0,), (2,), (0, 2), (1, 2)]:
        a = oracle_mod.fmo_fragment_integrals(t["h"], t["eri"], t["frag_orbs"], t["frag_nocc"],
                                              members)
        b = serving.fmo_fragment_integrals(t["h"], t["eri"], t["frag_orbs"], t["frag_nocc"],
                                           members)
        assert a[2] == b[2]
        assert np.max(np.abs(a[0] - b[0])) < 1e-12 and np.max(np.abs(a[1] - b[1])) < 1e-14
