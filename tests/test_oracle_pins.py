"""Pins of the CPU oracle against things other than itself.

Each test fixes part of the oracle by an independent construction, a closed
form, a library routine or an exact invariant of the method (paper
Sections 2.2-3.2, Eqs. 2-6).  A plausible slip in the oracle (a dropped
term, a wrong sign, a transposed index, a wrong operator order) fails at
least one of them.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import synth
from tests import _dense

TOL = 1e-12


def small_case(n_orb=4, n_chol=6, seed=0):
    h, eri, e_core = synth.make_integrals(n_orb, n_chol, seed)
    return h, eri, e_core


def closed_shell_hf(h, eri, n_occ):
    """Textbook closed-shell HF energy in spatial orbitals:
    E = 2 sum_i h_ii + sum_ij [2 (ii|jj) - (ij|ji)]."""
    e = 0.0
    for i in range(n_occ):
        e += 2.0 * h[i, i]
        for j in range(n_occ):
            e += 2.0 * eri[i, i, j, j] - eri[i, j, j, i]
    return e


# ---------------------------------------------------------------------------
# Hamiltonian (Eq. 2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["eq2", "sc"])
def test_h_apply_matches_dense_kronecker_jw(oracle_mod, method):
    n_orb = 4
    h, eri, _ = small_case(n_orb)
    e_core = 0.37
    H = _dense.hamiltonian(n_orb, h, eri, e_core)
    psi = synth.random_state(2 * n_orb, seed=11)  # all sectors populated
    sig = oracle_mod.h_apply(n_orb, h, eri, e_core, psi, method)
    ref = H @ psi
    assert np.max(np.abs(sig - ref)) < TOL


def test_sc_matches_eq2_12q(oracle_mod):
    n_orb = 6
    h, eri, e_core = small_case(n_orb, 10, 1)
    n = 2 * n_orb
    psi = synth.random_state(n, seed=5, sector=lambda x: bin(x).count("1") == 6)
    a = oracle_mod.h_apply(n_orb, h, eri, e_core, psi, "eq2")
    b = oracle_mod.h_apply(n_orb, h, eri, e_core, psi, "sc")
    assert np.max(np.abs(a - b)) < 1e-11


def test_hf_energy_closed_form(oracle_mod):
    for (n_orb, n_chol, seed, n_e) in [(4, 6, 0, 4), (6, 10, 1, 6), (5, 3, 9, 4)]:
        h, eri, e_core = synth.make_integrals(n_orb, n_chol, seed)
        ex = oracle_mod.excitations(n_orb, n_e // 2, n_e // 2)
        E, g = oracle_mod.energy_grad(n_orb, h, eri, e_core, n_e // 2, n_e // 2, ex,
                                      np.zeros(len(ex)))
        assert abs(E - closed_shell_hf(h, eri, n_e // 2)) < 1e-11


def test_hamiltonian_hermitian_and_conserving(oracle_mod):
    n_orb = 4
    h, eri, e_core = small_case(n_orb)
    Hs, basis = oracle_mod.h_sector_matrix(n_orb, h, eri, e_core, 2, 2, "eq2")
    assert np.max(np.abs(Hs - Hs.T)) < TOL
    # H psi stays in the sector (particle number and S_z conserved).
    n = 2 * n_orb
    inside = np.zeros(1 << n, dtype=bool)
    inside[basis] = True
    psi = np.zeros(1 << n, dtype=complex)
    psi[basis] = synth.random_state(n, 3)[basis]
    sig = oracle_mod.h_apply(n_orb, h, eri, e_core, psi, "eq2")
    assert np.max(np.abs(sig[~inside])) == 0.0


def test_fci_matches_dense_kronecker(oracle_mod):
    n_orb = 4
    h, eri, e_core = small_case(n_orb)
    H = _dense.hamiltonian(n_orb, h, eri, e_core).toarray()
    basis = oracle_mod.sector_basis(8, 2, 2)
    e_ref = np.linalg.eigvalsh(H[np.ix_(basis, basis)])[0]
    assert abs(oracle_mod.fci_energy(n_orb, h, eri, e_core, 2, 2) - e_ref) < 1e-11


# ---------------------------------------------------------------------------
# Generators and rotations (Eq. 4, Eq. 5)
# ---------------------------------------------------------------------------
def test_excitation_counts(oracle_mod):
    # closed form: singles 2 * o * v, doubles 2*C(o,2)*C(v,2) + (o*v)^2 per
    # spin-orbital occupied/virtual counts o, v of each spin.
    for n_orb, n_e, K in [(4, 4, 26), (6, 6, 117), (9, 10, 560), (13, 12, 2478)]:
        o = n_e // 2
        v = n_orb - o
        closed = 2 * o * v + 2 * math.comb(o, 2) * math.comb(v, 2) + (o * v) ** 2
        ex = oracle_mod.excitations(n_orb, o, o)
        assert len(ex) == K == closed
        singles = ex[ex[:, 1] < 0]
        assert len(singles) == 2 * o * v
        # lexicographic within singles and doubles
        d = [tuple(r) for r in ex[ex[:, 1] >= 0]]
        assert d == sorted(d)
        s = [tuple(r) for r in singles]
        assert s == sorted(s)


def test_generator_matches_dense(oracle_mod):
    n = 8
    ex = oracle_mod.excitations(4, 2, 2)
    psi = synth.random_state(n, 21)
    for row in ex[::3]:
        G = _dense.generator(n, row)
        assert np.max(np.abs(oracle_mod.apply_generator(n, row, psi) - G @ psi)) < TOL
        # G is real antisymmetric and G^3 = -G
        assert np.max(np.abs(G + G.T)) == 0.0
        assert np.max(np.abs(G @ G @ G + G)) < TOL


def test_rotation_matches_expm(oracle_mod):
    n = 8
    ex = oracle_mod.excitations(4, 2, 2)
    psi = synth.random_state(n, 22)
    for row, phi in zip(ex[::2], np.linspace(-2.5, 2.9, len(ex[::2]))):
        G = _dense.generator(n, row)
        ref = scipy.linalg.expm(phi * G) @ psi
        got = oracle_mod.rotate(n, row, phi, psi)
        assert np.max(np.abs(got - ref)) < 1e-12
        back = oracle_mod.rotate(n, row, -phi, got)
        assert np.max(np.abs(back - psi)) < 1e-12


def _pauli_expansion(M, n):
    out = []
    for labels in itertools.product("IXYZ", repeat=n):
        P = _dense.pauli_string(labels)
        c = np.trace(P.conj().T @ M) / (1 << n)
        if abs(c) > 1e-14:
            out.append((c, P))
    return out


@pytest.mark.parametrize("row", [(0, -1, 2, -1), (1, -1, 3, -1), (0, 1, 2, 3), (0, 1, 4, 5),
                                 (1, 3, 4, 5)])
def test_rotation_equals_product_of_pauli_exponentials(oracle_mod, row):
    """The paper Trotterises Pauli strings, exp(i t_k P_k) (Eq. 5); the JW
    strings of one excitation commute, so their product in any order is
    exp(theta G).  Checked against the oracle's rotation on 6 qubits."""
    n = 6
    G = _dense.generator(n, row)
    theta = 0.731
    terms = _pauli_expansion(theta * G, n)  # theta G = sum_P (i t_P) P
    assert len(terms) in (2, 8)
    psi = synth.random_state(n, 4)
    for perm in (terms, terms[::-1]):
        U = np.eye(1 << n, dtype=complex)
        for c, P in perm:
            U = scipy.linalg.expm(c * P) @ U
        got = oracle_mod.rotate(n, np.array(row, dtype=np.int32), theta, psi)
        assert np.max(np.abs(U @ psi - got)) < 1e-13


def test_full_ansatz_matches_ordered_expm_product(oracle_mod):
    n_orb = 4
    h, eri, e_core = small_case(n_orb)
    ex = oracle_mod.excitations(n_orb, 2, 2)
    theta = synth.theta_uniform(len(ex), -0.4, 0.4, 1000)
    E, _, psi, sig = oracle_mod.energy_grad(n_orb, h, eri, e_core, 2, 2, ex, theta,
                                             grad=False, want_state=True)
    ref = np.zeros(256, dtype=complex)
    ref[oracle_mod.hf_index(2, 2)] = 1.0
    for k, row in enumerate(ex):  # excitation 1 acts first
        ref = scipy.linalg.expm(theta[k] * _dense.generator(8, row)) @ ref
    assert np.max(np.abs(psi - ref)) < 1e-12
    H = _dense.hamiltonian(n_orb, h, eri, e_core)
    assert abs(E - np.vdot(ref, H @ ref).real) < 1e-12


@pytest.mark.parametrize("name", ["8q", "12q"])
def test_state_invariants(oracle_mod, name):
    w = synth.workload(name)
    n = 2 * w["n_orb"]
    ex = oracle_mod.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
    theta = synth.theta_normal(len(ex), 0.3, 77)
    E, _, psi, _ = oracle_mod.energy_grad(w["n_orb"], w["h"], w["eri"], w["e_core"],
                                          w["n_alpha"], w["n_beta"], ex, theta,
                                          grad=False, want_state=True)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-13
    p = np.abs(psi) ** 2
    assert abs(p @ _dense.number_op(n) - w["n_elec"]) < 1e-12
    assert abs(p @ _dense.sz_op(n)) < 1e-12
    assert np.max(np.abs(psi.imag)) == 0.0
    e_fci = oracle_mod.fci_energy(w["n_orb"], w["h"], w["eri"], w["e_core"],
                                  w["n_alpha"], w["n_beta"])
    assert E >= e_fci - 1e-12


def test_energy_trig_structure_along_one_amplitude(oracle_mod):
    """E(theta0 + phi e_k) is a trigonometric polynomial of degree 2 in phi
    (spectrum of G_k is {0, +i, -i}); on the 16-point sweep the DFT content
    at frequencies 3..8 vanishes."""
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    theta0 = synth.theta_uniform(len(ex), -0.1, 0.1, 1000)
    k = int(np.nonzero(ex[:, 1] >= 0)[0][0])  # first double
    es = []
    for s in range(16):
        th = theta0.copy()
        th[k] += -math.pi + 2 * math.pi * s / 16
        es.append(oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, th, grad=False)[0])
    F = np.fft.rfft(np.array(es)) / 16
    assert np.max(np.abs(F[3:])) < 1e-12
    assert np.max(np.abs(F[1:3])) > 1e-6


@pytest.mark.parametrize("name", ["8q", "12q"])
def test_adjoint_gradient_fd_and_fourier(oracle_mod, name):
    w = synth.workload(name)
    no = w["n_orb"]
    ex = oracle_mod.excitations(no, w["n_alpha"], w["n_beta"])
    theta = synth.theta_normal(len(ex), 0.2, 31)
    args = (no, w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"], ex)
    E, g = oracle_mod.energy_grad(*args, theta)
    ks = range(len(ex)) if name == "8q" else range(0, len(ex), 13)
    for k in ks:
        # exact Fourier derivative: 5 samples at phi in {0, +-2pi/5, +-4pi/5}
        phis = [2 * math.pi * m / 5 for m in range(5)]
        es = []
        for phi in phis:
            th = theta.copy()
            th[k] += phi
            es.append(oracle_mod.energy_grad(*args, th, grad=False)[0])
        # E(phi) = a0 + sum_{m=1,2} a_m cos(m phi) + b_m sin(m phi)
        b = [2.0 / 5 * sum(e * math.sin(m * p) for e, p in zip(es, phis)) for m in (1, 2)]
        d_fourier = b[0] + 2 * b[1]
        assert abs(g[k] - d_fourier) < 1e-10
        hstep = 1e-4
        tp, tm = theta.copy(), theta.copy()
        tp[k] += hstep
        tm[k] -= hstep
        fd = (oracle_mod.energy_grad(*args, tp, grad=False)[0]
              - oracle_mod.energy_grad(*args, tm, grad=False)[0]) / (2 * hstep)
        assert abs(g[k] - fd) < 1e-7


def test_gradient_with_slices_and_second_order(oracle_mod):
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    theta = synth.theta_normal(len(ex), 0.3, 41)
    args = (4, w["h"], w["eri"], 0.0, 2, 2, ex)
    for order, M in [(1, 3), (2, 1), (2, 2)]:
        _, g = oracle_mod.energy_grad(*args, theta, order=order, M=M)
        for k in (0, 9, 25):
            hstep = 1e-4
            tp, tm = theta.copy(), theta.copy()
            tp[k] += hstep
            tm[k] -= hstep
            fd = (oracle_mod.energy_grad(*args, tp, order=order, M=M, grad=False)[0]
                  - oracle_mod.energy_grad(*args, tm, order=order, M=M, grad=False)[0]) / (2 * hstep)
            assert abs(g[k] - fd) < 1e-7


# ---------------------------------------------------------------------------
# Trotter structure (Eq. 5, Eq. 6)
# ---------------------------------------------------------------------------
def test_order_matters(oracle_mod):
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    theta = synth.theta_normal(len(ex), 0.3, 8)
    E1, _ = oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta, grad=False)
    E2, _ = oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex[::-1].copy(),
                                   theta[::-1].copy(), grad=False)
    assert abs(E1 - E2) > 1e-6


def test_disjoint_excitations_commute_and_are_trotter_exact(oracle_mod):
    w = synth.workload("8q")
    ex = np.array([(0, -1, 4, -1), (1, 3, 5, 7), (2, -1, 6, -1)], dtype=np.int32)
    theta = np.array([0.41, -0.77, 0.29])
    a = oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta, grad=False)[0]
    perm = [2, 0, 1]
    b = oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex[perm].copy(),
                               theta[perm].copy(), grad=False)[0]
    c, _ = oracle_mod.trotter_free_energy(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta)
    assert abs(a - b) < 1e-13 and abs(a - c) < 1e-12


def test_single_excitation_trotter_any_M_is_exact(oracle_mod):
    w = synth.workload("8q")
    ex = np.array([(1, 3, 5, 7)], dtype=np.int32)
    theta = np.array([0.93])
    c, _ = oracle_mod.trotter_free_energy(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta)
    for order, M in [(1, 1), (1, 3), (2, 2)]:
        a = oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta,
                                   order=order, M=M, grad=False)[0]
        assert abs(a - c) < 1e-12


def test_trotter_error_shrinks_with_slices_and_second_order(oracle_mod):
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    theta = synth.theta_normal(len(ex), 0.25, 12)
    ref, _ = oracle_mod.trotter_free_energy(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta)
    err1 = [abs(oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta, order=1,
                                       M=M, grad=False)[0] - ref) for M in (1, 2, 4, 8)]
    err2 = abs(oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta, order=2,
                                      M=1, grad=False)[0] - ref)
    assert err1[0] > err1[1] > err1[2] > err1[3]
    assert err2 < err1[0]


# ---------------------------------------------------------------------------
# Paper-motivated invariants (Section 3.2)
# ---------------------------------------------------------------------------
def test_orbital_sign_gauge(oracle_mod):
    """Flipping the sign of spatial orbital p in h and (pq|rs) and of every
    theta_k whose indices hit p an odd number of times leaves the Trotterised
    energy unchanged (the phase effect discussed in Section 3.2)."""
    w = synth.workload("12q")
    no = 6
    ex = oracle_mod.excitations(no, 3, 3)
    theta = synth.theta_normal(len(ex), 0.3, 17)
    E, g = oracle_mod.energy_grad(no, w["h"], w["eri"], 0.0, 3, 3, ex, theta)
    for p in (1, 4):
        s = np.ones(no)
        s[p] = -1.0
        h2 = w["h"] * s[:, None] * s[None, :]
        eri2 = w["eri"] * np.einsum("p,q,r,s->pqrs", s, s, s, s)
        par = np.array([sum(1 for v in row if v >= 0 and v // 2 == p) % 2 for row in ex])
        th2 = theta * np.where(par == 1, -1.0, 1.0)
        E2, g2 = oracle_mod.energy_grad(no, h2, eri2, 0.0, 3, 3, ex, th2)
        assert abs(E - E2) < 1e-11
        assert np.max(np.abs(np.abs(g) - np.abs(g2))) < 1e-10


def test_size_consistency_local_fragments(oracle_mod):
    """Two non-interacting fragments with orbitals ordered [A_occ, B_occ,
    A_virt, B_virt] and only intra-fragment excitations: the Trotterised
    dimer energy is E_A + E_B exactly (Section 3.2, Table 6 LMO rows)."""
    hA, eA, _ = synth.make_integrals(3, 4, 101)
    hB, eB, _ = synth.make_integrals(3, 4, 202)
    # dimer orbital order: A0, B0, A1, A2, B1, B2  (A0, B0 occupied)
    A = [0, 2, 3]
    B = [1, 4, 5]
    h = np.zeros((6, 6))
    eri = np.zeros((6,) * 4)
    h[np.ix_(A, A)] = hA
    h[np.ix_(B, B)] = hB
    eri[np.ix_(A, A, A, A)] = eA
    eri[np.ix_(B, B, B, B)] = eB
    exA = oracle_mod.excitations(3, 1, 1)
    exB = oracle_mod.excitations(3, 1, 1)
    thA = synth.theta_normal(len(exA), 0.5, 5)
    thB = synth.theta_normal(len(exB), 0.5, 6)

    def remap(row, orbs):
        return tuple(-1 if v < 0 else 2 * orbs[v // 2] + v % 2 for v in row)

    rows = [remap(r, A) for r in exA] + [remap(r, B) for r in exB]
    th = np.concatenate([thA, thB])
    EA = oracle_mod.energy_grad(3, hA, eA, 0.0, 1, 1, exA, thA, grad=False)[0]
    EB = oracle_mod.energy_grad(3, hB, eB, 0.0, 1, 1, exB, thB, grad=False)[0]
    ED = oracle_mod.energy_grad(6, h, eri, 0.0, 2, 2, np.array(rows, dtype=np.int32), th,
                                grad=False)[0]
    assert abs(ED - (EA + EB)) < 1e-11


def test_sector_mode_equals_full_mode(oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    theta = synth.theta_normal(len(ex), 0.2, 3)
    a = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, theta, sector=False)
    b = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, theta, sector=True)
    assert abs(a[0] - b[0]) < 1e-12
    assert np.max(np.abs(a[1] - b[1])) < 1e-12
    c = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, theta, method="eq2")
    assert abs(a[0] - c[0]) < 1e-11
    assert np.max(np.abs(a[1] - c[1])) < 1e-11


def test_sector_sizes(oracle_mod):
    assert oracle_mod.sector_size(8, 2, 2) == 36
    assert oracle_mod.sector_size(12, 3, 3) == 400
    assert oracle_mod.sector_size(18, 5, 5) == 15876
