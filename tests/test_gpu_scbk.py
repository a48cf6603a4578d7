"""The state held in the tapered symmetry-conserving Bravyi-Kitaev encoding
(UCCSD_LAYOUT_SCBK, the paper's qubit counts, Section 2.3): n - 2 qubits.

Energies and gradients equal the oracle's Jordan-Wigner values to 1e-10
(FP64) and the 2^n layout's bitwise; the exported 2^(n-2) state, acted on
by the tapered Hamiltonian that uccsd_pauli_terms_scbk compiles on the host
(a separate compile from the one the kernels use), gives the oracle's energy
and has norm 1, so the device state is the paper's encoding of |Psi>."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def uc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_17993_gb300 as uc
    uc.lib()
    return uc


def _apply_paulis(x, z, c, psi):
    """sum_t c_t X^{x_t} Z^{z_t} psi with X^x Z^z |b> = (-1)^{popc(b & z)} |b ^ x>."""
    b = np.arange(psi.size, dtype=np.uint32)
    out = np.zeros_like(psi)
    for xt, zt, ct in zip(x, z, c):
        par = np.bitwise_count(b & zt) & 1 if hasattr(np, "bitwise_count") else \
            np.array([bin(int(v)).count("1") & 1 for v in (b & zt)])
        out[b ^ xt] += ct * np.where(par, -1.0, 1.0) * psi
    return out


@pytest.mark.parametrize("name", ["8q", "12q"])
def test_tapered_state_gives_the_oracle_energy(uc, oracle_mod, name):
    w = synth.workload(name)
    ex = oracle_mod.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
    th = synth.theta_uniform(len(ex), -0.1, 0.1, 1000)
    E0, g0 = oracle_mod.energy_grad(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"],
                                    w["n_beta"], ex, th)
    ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                          precision=uc.FP64, layout=uc.LAYOUT_SCBK)
    assert abs(ctx.energy(th) - E0) <= 1e-10
    psi = ctx.state(0)
    n = 2 * w["n_orb"]
    assert psi.size == 1 << (n - 2)
    assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-12
    x, z, c, nq = uc.pauli_terms_scbk(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"],
                                      w["n_beta"])
    assert nq == n - 2
    E_scbk = np.vdot(psi, _apply_paulis(x, z, c, psi)).real
    assert abs(E_scbk - E0) <= 1e-10
    E, g = ctx.energy_grad(th)
    assert abs(E - E0) <= 1e-10 and np.max(np.abs(g - g0)) <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_tapered_layout_is_bitwise_the_full_layout_at_18q(uc, prec):
    gold = json.load(open(os.path.join(HERE, "golden", "golden_18q.json")))
    w = synth.workload("18q")
    ctx = {lay: uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"],
                                w["n_beta"], precision=prec, layout=lay)
           for lay in (uc.LAYOUT_FULL, uc.LAYOUT_SCBK)}
    assert ctx[uc.LAYOUT_SCBK].info()["layout"] == uc.LAYOUT_SCBK
    tol = 1e-10 if prec == 0 else 1e-5
    for r in gold["evals"][:2]:
        th = synth.theta_normal(gold["K"], 0.05, r["theta_seed"])
        Ef, gf = ctx[uc.LAYOUT_FULL].energy_grad(th)
        Et, gt = ctx[uc.LAYOUT_SCBK].energy_grad(th)
        assert Ef == Et and np.array_equal(gf, gt)
        assert abs(Et - r["E"]) <= tol and np.max(np.abs(gt - np.array(r["grad"]))) <= tol
