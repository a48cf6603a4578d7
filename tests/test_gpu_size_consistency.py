"""Size consistency and orbital invariance of VQE-UCCSD (Section 3.2,
Tables 6 and S3) on synthetic non-interacting fragments, on the GPU.

A dimer of two identical fragments with no integral between them is solved
in localised orbitals (each orbital on one fragment) and in delocalised
orbitals (the symmetric/antisymmetric combinations, the canonical orbitals of
such a dimer).  The Trotter-free ansatz spans the same operator space in both
bases, so its VQE energy is basis independent and twice the monomer's; the
first-order Trotter product is not, and loses size consistency in the
delocalised basis.  Slices M = 1..5 shrink that error, and the fit
E = alpha (1/M)^beta + gamma extrapolates towards the Trotter-free value."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_17993_gb300 as uc
    uc.lib()
    return uc


@pytest.fixture(scope="module")
def frags():
    # weakly correlated fragment (off-diagonal h x0.1, Cholesky vectors x0.5):
    # UCCSD lands about 1 kcal/mol above FCI, as for the paper's H4 monomer
    h, eri, _ = synth.make_integrals(4, 6, 0, offdiag=0.1, chol=0.5)
    hd, ed, _ = synth.non_interacting_dimer(h, eri, 2, h, eri, 2)
    hc, ec = synth.rotate_orbitals(hd, ed, synth.pair_mixing(2, 2))
    return dict(mono=(h, eri), lmo=(hd, ed), cmo=(hc, ec))


def _vqe(uc, h, eri, n_orb, n_el, free=False, M=1, order=1):
    from paper_2402_17993_gb300 import vqe
    ctx = uc.make_context(n_orb, h, eri, 0.0, n_el, n_el, trotter_order=order, n_slices=M)
    E, th, n_eval, gn = vqe.minimize(ctx, gtol=1e-7, maxiter=4000, trotter_free=free)
    ctx.close()
    return E, th, gn


def test_localised_dimer_at_the_product_amplitudes_is_exactly_twice_the_monomer(uc, frags):
    h, eri = frags["mono"]
    E_a, th_a, _ = _vqe(uc, h, eri, 4, 2)
    mono = uc.build_uccsd_list(4, 2, 2)
    dim = uc.build_uccsd_list(8, 4, 4)
    # map monomer spin orbitals to fragment A (occ 0..3, virt 8..11) and B (occ 4..7, virt 12..15)
    def to_a(q):
        return q if q < 4 else q + 4
    def to_b(q):
        return q + 4 if q < 4 else q + 8
    index = {tuple(r): k for k, r in enumerate(dim.tolist())}
    th = np.zeros(len(dim))
    for k, r in enumerate(mono.tolist()):
        for f in (to_a, to_b):
            key = tuple(f(q) if q >= 0 else -1 for q in r)
            th[index[key]] = th_a[k]
    hd, ed = frags["lmo"]
    ctx = uc.make_context(8, hd, ed, 0.0, 4, 4)
    assert abs(ctx.energy(th) - 2 * E_a) < 1e-10
    # the same for the Trotter-free ansatz: exp(A_A + A_B) = exp(A_A) exp(A_B)
    cm = uc.make_context(4, h, eri, 0.0, 2, 2)
    assert abs(ctx.energy_trotter_free(th) - 2 * cm.energy_trotter_free(th_a)) < 1e-10
    cm.close()
    ctx.close()


def test_size_consistency_and_orbital_invariance_table(uc, oracle_mod, frags):
    h, eri = frags["mono"]
    hd, ed = frags["lmo"]
    hc, ec = frags["cmo"]
    e_fci = 2 * oracle_mod.fci_energy(4, h, eri, 0.0, 2, 2)
    r = {}
    r["mono"] = _vqe(uc, h, eri, 4, 2)[0]
    r["mono_free"] = _vqe(uc, h, eri, 4, 2, free=True)[0]
    r["lmo"] = _vqe(uc, hd, ed, 8, 4)[0]
    r["cmo"] = _vqe(uc, hc, ec, 8, 4)[0]
    r["lmo_free"] = _vqe(uc, hd, ed, 8, 4, free=True)[0]
    r["cmo_free"] = _vqe(uc, hc, ec, 8, 4, free=True)[0]
    cmo_M = [r["cmo"]] + [_vqe(uc, hc, ec, 8, 4, M=M)[0] for M in (2, 3, 4, 5)]
    r["cmo_2nd"] = _vqe(uc, hc, ec, 8, 4, order=2)[0]
    a, b, c = uc.trotter_extrapolate([1, 2, 3, 4, 5], cmo_M)
    kcal = 627.5095
    print("\nsize consistency, synthetic 4-orbital fragments (dimer minus twice the monomer, kcal/mol):")
    print(f"  Trotter M=1  localised {(r['lmo'] - 2 * r['mono']) * kcal:+.6f}  "
          f"delocalised {(r['cmo'] - 2 * r['mono']) * kcal:+.6f}")
    print(f"  Trotter-free localised {(r['lmo_free'] - 2 * r['mono_free']) * kcal:+.6f}  "
          f"delocalised {(r['cmo_free'] - 2 * r['mono_free']) * kcal:+.6f}")
    print("  delocalised, energy above FCI (kcal/mol) for M=1..5:",
          " ".join(f"{(e - e_fci) * kcal:.4f}" for e in cmo_M),
          f" 2nd order {(r['cmo_2nd'] - e_fci) * kcal:.4f}",
          f" Trotter-free {(r['cmo_free'] - e_fci) * kcal:.4f}")
    print(f"  fit alpha={a:.6g} beta={b:.4f} gamma-E_free={(c - r['cmo_free']) * 1e6:.1f} microhartree")
    for v in r.values():
        assert v >= e_fci - 1e-9
    # the Trotter-free ansatz is orbital invariant and (to a microhartree)
    # size consistent; so is the Trotter product in localised orbitals
    assert abs(r["cmo_free"] - r["lmo_free"]) < 1e-6
    assert abs(r["lmo_free"] - 2 * r["mono_free"]) < 1e-6
    assert abs(r["lmo"] - 2 * r["mono"]) < 1e-6
    # the Trotter product in delocalised orbitals is not, and slices reduce the error
    assert r["cmo"] - 2 * r["mono"] > 1e-5
    assert abs(cmo_M[-1] - r["cmo_free"]) < abs(cmo_M[0] - r["cmo_free"])
