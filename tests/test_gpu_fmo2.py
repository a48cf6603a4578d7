"""FMO two-body assembly (Section 2.1, Eq. 1) on a coherent synthetic
trimer: the six solves (three monomers at 8 qubits, three dimers at 16
qubits, each embedded in the other fragments' reference mean field) are
served by the fragment server, and Eq. 1 is assembled from their energies.

* Coupled fragments: every fragment energy at its served amplitudes equals
  the oracle's (own fragment integrals, own Hamiltonian action) to 1e-10, so
  the assembled totals agree.
* Non-interacting fragments: at the monomers' served amplitudes (cross-
  fragment amplitudes zero) every dimer energy on the device is the sum of
  its monomers', and the two-body total is the sum of the monomer energies."""
import itertools

import numpy as np
import pytest

import synth
from tests._fmo import dimer_theta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_17993_gb300 as uc
    uc.lib()
    return uc


def _energy(uc, q, theta):
    ctx = uc.make_context(q.n_orb, q.h, q.eri, q.e_core, q.n_alpha, q.n_beta, precision=uc.FP64)
    e = ctx.energy(theta)
    ctx.close()
    return e


def test_served_fmo2_total_matches_the_oracle(uc, oracle_mod):
    from paper_2402_17993_gb300 import serving
    t = synth.fmo_trimer(41, 0.3)
    reqs, keys = serving.fmo2_requests(t["h"], t["eri"], t["frag_orbs"], t["frag_nocc"])
    srv = serving.FragmentServer(precision=uc.FP64, steps=8, max_active=6)
    res, stats = srv.run(reqs, keep_theta=True)
    srv.close()
    assert stats["requests"] == 6
    gpu = [_energy(uc, q, r.theta) for q, r in zip(reqs, res)]
    mono, dim = {}, {}
    for key, q, r, e in zip(keys, reqs, res, gpu):
        hp, ep, nocc = oracle_mod.fmo_fragment_integrals(t["h"], t["eri"], t["frag_orbs"],
                                                         t["frag_nocc"], key)
        ex = oracle_mod.excitations(hp.shape[0], nocc, nocc)
        e_or = oracle_mod.energy_grad(hp.shape[0], hp, ep, 0.0, nocc, nocc, ex, r.theta,
                                      grad=False)[0]
        assert abs(e - e_or) <= 1e-10, key
        if len(key) == 1:
            mono[key[0]] = e_or
        else:
            dim[key] = e_or
        assert r.energies[-1] <= r.energies[0] + 1e-9  # the solve lowered the energy
    total_gpu = serving.fmo2_total(gpu, keys, 3)
    assert abs(total_gpu - oracle_mod.fmo2_energy(mono, dim, 3)) <= 1e-9


def test_non_interacting_fmo2_is_the_sum_of_monomers(uc, oracle_mod):
    from paper_2402_17993_gb300 import serving
    t = synth.fmo_trimer(42, 0.0)
    reqs, keys = serving.fmo2_requests(t["h"], t["eri"], t["frag_orbs"], t["frag_nocc"])
    srv = serving.FragmentServer(precision=uc.FP64, steps=8, max_active=6)
    res, _ = srv.run(reqs[:3], keep_theta=True)   # the monomer solves
    srv.close()
    mono = {k[0]: _energy(uc, q, r.theta) for k, q, r in zip(keys[:3], reqs[:3], res)}
    exs = {k[0]: uc.build_uccsd_list(q.n_orb, q.n_alpha, q.n_beta)
           for k, q in zip(keys[:3], reqs[:3])}
    thetas = {k[0]: r.theta for k, r in zip(keys[:3], res)}
    energies = [mono[i] for i in range(3)]
    for key, q in zip(keys[3:], reqs[3:]):
        i, j = key
        ex_d = uc.build_uccsd_list(q.n_orb, q.n_alpha, q.n_beta)
        nocc, nvir = t["frag_nocc"][i], len(t["frag_orbs"][i]) - t["frag_nocc"][i]
        th = dimer_theta(exs[i], thetas[i], exs[j], thetas[j], ex_d, nocc, nvir)
        e = _energy(uc, q, th)
        assert abs(e - mono[i] - mono[j]) <= 1e-10, key
        energies.append(e)
    assert abs(serving.fmo2_total(energies, keys, 3) - sum(mono.values())) <= 1e-10
