"""Pins of the oracle's Trotter-schedule helpers: the magnitude ordering of
Section 2.3 (with first-order amplitudes as the magnitudes) and the
Trotter-error extrapolation of Section 3.2 (Fig. 3).  CPU only."""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_extrapolation_reproduces_the_papers_fit_of_table_s3(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "table_s3_trotter_fit.json")))
    a, b, c = oracle_mod.trotter_extrapolate(g["M"], g["dE_kcal"])
    kc = g["kcal_per_hartree"]
    pf = g["paper_fit"]
    # inputs are printed to 1e-4 kcal/mol, the fit to 4-5 digits
    assert abs(a / kc - pf["alpha_hartree"]) < 2e-6
    assert abs(b - pf["beta"]) < 1e-3
    assert abs((c - g["expm_kcal"]) / kc * 1e6 - pf["gamma_minus_expm_microhartree"]) < 1.0


def test_extrapolation_recovers_an_exact_power_law(oracle_mod):
    M = np.arange(1, 6)
    for alpha, beta, gamma in [(0.3, 1.0, -2.0), (-0.01, 2.0, 5.0), (0.005396, 3.6466, -3.876244)]:
        E = alpha * (1.0 / M) ** beta + gamma
        a, b, c = oracle_mod.trotter_extrapolate(M, E)
        assert abs(a - alpha) < 1e-9 * max(1, abs(alpha)) + 1e-12
        assert abs(b - beta) < 1e-6
        assert abs(c - gamma) < 1e-10 * max(1, abs(gamma))


def _det_energy(oracle_mod, n_orb, w, x):
    e = np.zeros(1 << (2 * n_orb), dtype=np.complex128)
    e[x] = 1.0
    return oracle_mod.h_apply(n_orb, w["h"], w["eri"], 0.0, e)[x].real


def test_fock_diagonal_is_the_difference_of_determinant_energies(oracle_mod):
    # eps_a = <HF+a|H|HF+a> - <HF|H|HF> (virtual), eps_i = <HF|H|HF> - <HF-i|H|HF-i>
    w = synth.workload("8q")
    n_orb, na, nb = 4, 2, 2
    hf = oracle_mod.hf_index(na, nb)
    eps = oracle_mod.fock_diagonal(n_orb, w["h"], w["eri"], na, nb)
    e0 = _det_energy(oracle_mod, n_orb, w, hf)
    for P in range(2 * n_orb):
        e1 = _det_energy(oracle_mod, n_orb, w, hf ^ (1 << P))
        want = (e1 - e0) if not (hf >> P) & 1 else (e0 - e1)
        assert abs(eps[P] - want) < 1e-12


@pytest.mark.parametrize("name,na", [("8q", 2), ("12q", 3)])
def test_mp1_amplitudes_give_the_textbook_closed_shell_mp2_sums(oracle_mod, name, na):
    # sum_k t_k <Phi_k|H|HF> over doubles = sum_ijab (ia|jb)[2(ia|jb)-(ib|ja)]/D_ijab
    # (closed-shell spatial-orbital form); over singles = 2 sum_ia f_ia^2/(e_i-e_a)
    w = synth.workload(name)
    n_orb = w["n_orb"]
    h, eri = w["h"], w["eri"]
    ex = oracle_mod.excitations(n_orb, na, na)
    t, num = oracle_mod.mp1_amplitudes(n_orb, h, eri, 0.0, na, na, ex)
    occ, vir = range(na), range(na, n_orb)
    e = np.array([h[p, p] + sum(2 * eri[p, p, j, j] - eri[p, j, j, p] for j in occ)
                  for p in range(n_orb)])
    f = lambda p, q: h[p, q] + sum(2 * eri[p, q, j, j] - eri[p, j, j, q] for j in occ)
    e2d = sum(eri[i, a, j, b] * (2 * eri[i, a, j, b] - eri[i, b, j, a]) / (e[i] + e[j] - e[a] - e[b])
              for i in occ for j in occ for a in vir for b in vir)
    e2s = 2 * sum(f(i, a) ** 2 / (e[i] - e[a]) for i in occ for a in vir)
    single = ex[:, 1] < 0
    assert abs(np.sum(t[~single] * num[~single]) - e2d) < 1e-12 * max(1, abs(e2d))
    assert abs(np.sum(t[single] * num[single]) - e2s) < 1e-12 * max(1, abs(e2s))


def test_mp1_numerator_is_half_the_energy_slope_at_zero(oracle_mod):
    # dE/dtheta_k at theta = 0 is 2 <HF|H tau_k|HF>; central difference, step 1e-4
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    _, num = oracle_mod.mp1_amplitudes(4, w["h"], w["eri"], 0.0, 2, 2, ex)
    hstep = 1e-4
    for k in (0, 3, 9, len(ex) - 1):
        th = np.zeros(len(ex))
        th[k] = hstep
        ep = oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, th, grad=False)[0]
        th[k] = -hstep
        em = oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, th, grad=False)[0]
        assert abs((ep - em) / (2 * hstep) - 2 * num[k]) < 1e-7


def test_magnitude_order_by_brute_force(oracle_mod):
    rows = np.arange(28, dtype=np.int32).reshape(7, 4)
    t = np.array([0.1, -0.3, 0.3, 0.0, -0.1, 2.0, 0.3])
    out, perm = oracle_mod.magnitude_order(rows, t)
    assert list(perm) == [5, 1, 2, 6, 0, 4, 3]  # |t| descending, ties in list order
    assert np.array_equal(out, rows[perm])


@pytest.mark.parametrize("order,beta", [(1, 1.0), (2, 2.0)])
def test_fixed_theta_trotter_error_has_the_product_formula_order(oracle_mod, order, beta):
    # at fixed theta the first-order product (Eq. 5) converges as 1/M and the
    # symmetric second-order one (Eq. 6) as 1/M^2 to exp(sum theta G)|HF>;
    # the fit's gamma lands far closer to that limit than E(M = 5) does
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    th = synth.theta_normal(len(ex), 0.05, 1000)
    E_free, _ = oracle_mod.trotter_free_energy(4, w["h"], w["eri"], 0.0, 2, 2, ex, th)
    Ms = [1, 2, 3, 4, 5]
    Es = [oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, th, order=order, M=M,
                                 grad=False)[0] for M in Ms]
    a, b, c = oracle_mod.trotter_extrapolate(Ms, Es)
    assert abs(b - beta) < 0.1 * beta
    assert abs(c - E_free) < 0.1 * abs(Es[-1] - E_free)


# --- Trotter-free ansatz on the sector (Eq. 3, Section 3.2's expm_multiply reference) ---

def test_sector_generator_sum_is_the_dense_sum_restricted_to_the_sector(oracle_mod):
    ex = oracle_mod.excitations(4, 2, 2)
    th = synth.theta_normal(len(ex), 0.3, 77)
    A = oracle_mod.generator_sum_sector(8, 2, 2, ex, th).toarray()
    dense = sum(th[k] * oracle_mod.generator_matrix(8, ex[k]) for k in range(len(ex)))
    basis = oracle_mod.sector_basis(8, 2, 2)
    assert np.array_equal(A, dense[np.ix_(basis, basis)])
    assert np.array_equal(A, -A.T)  # real antisymmetric: exp(A) is orthogonal


def test_sector_trotter_free_energy_equals_dense_expm(oracle_mod):
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    th = synth.theta_normal(len(ex), 0.3, 77)
    E1, p1 = oracle_mod.trotter_free_energy_sector(4, w["h"], w["eri"], 0.0, 2, 2, ex, th)
    E2, p2 = oracle_mod.trotter_free_energy(4, w["h"], w["eri"], 0.0, 2, 2, ex, th)
    assert abs(E1 - E2) < 1e-12 and np.max(np.abs(p1 - p2)) < 1e-13
    assert abs(np.linalg.norm(p1) - 1.0) < 1e-13


def test_trotter_free_equals_trotter_for_commuting_or_single_generators(oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    # generators on disjoint spin orbitals commute: the product is exact
    used, pick = set(), []
    for k, r in enumerate(ex):
        q = {int(v) for v in r if v >= 0}
        if not q & used:
            used |= q
            pick.append(k)
    sub = ex[pick]
    assert len(sub) >= 2
    for rows in (sub, ex[5:6], ex[40:41]):
        th = synth.theta_normal(len(rows), 0.4, 5)
        Ef, _ = oracle_mod.trotter_free_energy_sector(6, w["h"], w["eri"], 0.0, 3, 3, rows, th)
        Et = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, rows, th, grad=False)[0]
        assert abs(Ef - Et) < 1e-12


def test_trotter_energies_converge_to_the_trotter_free_energy(oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    th = synth.theta_normal(len(ex), 0.05, 1001)
    Ef, _ = oracle_mod.trotter_free_energy_sector(6, w["h"], w["eri"], 0.0, 3, 3, ex, th)
    e = [abs(oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, th, M=M, grad=False)[0] - Ef)
         for M in (1, 4, 16)]
    assert e[1] < e[0] / 3 and e[2] < e[1] / 3
    assert Ef >= oracle_mod.fci_energy(6, w["h"], w["eri"], 0.0, 3, 3) - 1e-12


def test_trotter_free_gradient_matches_central_differences(oracle_mod):
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    th = synth.theta_normal(len(ex), 0.3, 77)
    E, g = oracle_mod.trotter_free_energy_grad_sector(4, w["h"], w["eri"], 0.0, 2, 2, ex, th)
    E1, _ = oracle_mod.trotter_free_energy_sector(4, w["h"], w["eri"], 0.0, 2, 2, ex, th)
    assert abs(E - E1) < 1e-12
    hstep = 1e-5
    for k in range(len(ex)):
        tp, tm = th.copy(), th.copy()
        tp[k] += hstep
        tm[k] -= hstep
        ep = oracle_mod.trotter_free_energy_sector(4, w["h"], w["eri"], 0.0, 2, 2, ex, tp)[0]
        em = oracle_mod.trotter_free_energy_sector(4, w["h"], w["eri"], 0.0, 2, 2, ex, tm)[0]
        assert abs((ep - em) / (2 * hstep) - g[k]) < 1e-8


def test_trotter_free_gradient_equals_trotter_gradient_for_commuting_generators(oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    used, pick = set(), []
    for k, r in enumerate(ex):
        q = {int(v) for v in r if v >= 0}
        if not q & used:
            used |= q
            pick.append(k)
    sub = ex[pick]
    th = synth.theta_normal(len(sub), 0.4, 5)
    E, g = oracle_mod.trotter_free_energy_grad_sector(6, w["h"], w["eri"], 0.0, 3, 3, sub, th)
    Et, gt = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, sub, th)
    assert abs(E - Et) < 1e-12 and np.max(np.abs(g - gt)) < 1e-12
