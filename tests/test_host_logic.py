"""Host logic of the CUDA library, checked on the CPU (no device calls).

* the shared library loads and exports every symbol of include/uccsd.h;
* the excitation-list builder (Eq. 4) equals the oracle's list bit for bit;
* the Jordan-Wigner compile of Eq. 2 reproduces the X-mask group and Pauli
  term counts of dense synthetic integrals and, as a dense matrix, the
  Kronecker-product Jordan-Wigner Hamiltonian;
* invalid input is rejected with UCCSD_ERR_ARG.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import synth
from tests import _dense

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def uc():
    from paper_2402_17993_gb300 import build
    build.build()
    import paper_2402_17993_gb300 as uc
    return uc


def header_symbols():
    src = open(os.path.join(ROOT, "include", "uccsd.h")).read()
    return sorted(set(re.findall(r"\b(uccsd_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(uc):
    L = ctypes.CDLL(uc.LIB_PATH)
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(uc.EXPORTS) == syms


@pytest.mark.parametrize("n_orb,na,nb", [(4, 2, 2), (6, 3, 3), (9, 5, 5), (13, 6, 6), (5, 3, 1),
                                         (3, 0, 2), (2, 2, 2), (1, 1, 0)])
def test_excitation_list_matches_oracle(uc, oracle_mod, n_orb, na, nb):
    a = uc.build_uccsd_list(n_orb, na, nb)
    b = oracle_mod.excitations(n_orb, na, nb)
    assert a.shape == b.shape and np.array_equal(a, b)


def test_group_and_term_counts(uc):
    # groups: 1 + 2 C(n_orb,2) + 2 C(n_orb,4) + C(n_orb,2)^2 for dense integrals
    expect = {"8q": (51, 361), "12q": (286, 1819), "18q": (1621, 9316), "26q": (7671, 41068)}
    for name, (G, T) in expect.items():
        w = synth.workload(name)
        no = w["n_orb"]
        g, t = uc.hamiltonian_stats(no, w["h"], w["eri"], 0.0)
        closed = 1 + 2 * math.comb(no, 2) + 2 * math.comb(no, 4) + math.comb(no, 2) ** 2
        assert g == G == closed, name
        assert t == T, name


def xz_dense(n, x, z, c):
    N = 1 << n
    M = np.zeros((N, N))
    ys = np.arange(N)
    for xi, zi, ci in zip(x, z, c):
        sgn = np.array([-1.0 if bin(int(y) & int(zi)).count("1") % 2 else 1.0 for y in ys])
        M[ys ^ int(xi), ys] += ci * sgn
    return M


@pytest.mark.parametrize("n_orb,seed", [(3, 5), (4, 0)])
def test_pauli_terms_equal_dense_jordan_wigner(uc, n_orb, seed):
    h, eri, _ = synth.make_integrals(n_orb, n_orb + 2, seed)
    e_core = -1.25
    x, z, c = uc.pauli_terms(n_orb, h, eri, e_core)
    M = xz_dense(2 * n_orb, x, z, c)
    H = _dense.hamiltonian(n_orb, h, eri, e_core).toarray()
    assert np.max(np.abs(M - H)) < 1e-12
    # every Hermitian Pauli string with real coefficient has an even number of Y
    assert all(bin(int(a) & int(b)).count("1") % 2 == 0 for a, b in zip(x, z))


def test_invalid_hamiltonian_rejected(uc):
    h, eri, _ = synth.make_integrals(3, 4, 0)
    bad = h.copy()
    bad[0, 1] += 1e-6
    with pytest.raises(uc.UCCSDError) as e:
        uc.hamiltonian_stats(3, bad, eri)
    assert e.value.code == 1
    bad_eri = eri.copy()
    bad_eri[0, 1, 2, 2] += 1e-6
    with pytest.raises(uc.UCCSDError):
        uc.hamiltonian_stats(3, h, bad_eri)
    nan = h.copy()
    nan[1, 1] = float("nan")
    with pytest.raises(uc.UCCSDError):
        uc.hamiltonian_stats(3, nan, eri)
    with pytest.raises(uc.UCCSDError):
        uc.build_uccsd_list(16, 1, 1)


def test_status_strings(uc):
    L = uc.lib()
    for code in range(7):
        assert L.uccsd_status_string(code)


def test_magnitude_order_equals_oracle(uc, oracle_mod):
    # Section 2.3 ordering: same permutation as the oracle, ties included
    ex = oracle_mod.excitations(6, 3, 3)
    rng = np.random.default_rng(3)
    t = np.round(rng.normal(size=len(ex)), 1)  # rounding creates many ties, of both signs
    rows, perm = uc.magnitude_order(ex, t)
    want_rows, want_perm = oracle_mod.magnitude_order(ex, t)
    assert np.array_equal(perm, want_perm)
    assert np.array_equal(rows, want_rows)
    # aliasing output and input is allowed
    ex2 = np.ascontiguousarray(ex.copy())
    st = uc.lib().uccsd_magnitude_order(len(ex2), uc._i32p(ex2), uc._f64p(t), uc._i32p(ex2), None)
    assert st == 0 and np.array_equal(ex2, want_rows)


def test_magnitude_order_rejects_bad_input(uc):
    with pytest.raises(uc.UCCSDError):
        uc.magnitude_order(np.zeros((2, 4), np.int32), np.array([1.0, np.nan]))
    assert uc.lib().uccsd_magnitude_order(-1, None, None, None, None) == 1
    rows, perm = uc.magnitude_order(np.zeros((0, 4), np.int32), np.zeros(0))
    assert rows.shape == (0, 4) and perm.shape == (0,)


def test_trotter_extrapolation_equals_oracle_on_table_s3(uc, oracle_mod):
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "table_s3_trotter_fit.json")))
    got = uc.trotter_extrapolate(g["M"], g["dE_kcal"])
    want = oracle_mod.trotter_extrapolate(g["M"], g["dE_kcal"])
    assert abs(got[0] - want[0]) < 1e-6 * abs(want[0])
    assert abs(got[1] - want[1]) < 1e-6 * abs(want[1])
    assert abs(got[2] - want[2]) < 1e-8
    kc = g["kcal_per_hartree"]
    assert abs(got[0] / kc - g["paper_fit"]["alpha_hartree"]) < 2e-6
    assert abs(got[1] - g["paper_fit"]["beta"]) < 1e-3


@pytest.mark.parametrize("alpha,beta,gamma", [(0.3, 1.0, -2.0), (-0.01, 2.0, 5.0),
                                              (0.005396, 3.6466, -3.876244), (1e-6, 0.5, -75.0)])
def test_trotter_extrapolation_recovers_exact_power_laws(uc, alpha, beta, gamma):
    M = np.array([1, 2, 3, 4, 5, 6])
    E = alpha * (1.0 / M) ** beta + gamma
    a, b, c = uc.trotter_extrapolate(M, E)
    assert abs(b - beta) < 1e-5 * beta
    assert abs(a - alpha) < 1e-5 * abs(alpha)
    assert abs(c - gamma) < 1e-9 * max(1.0, abs(alpha))


def test_trotter_extrapolation_rejects_bad_input(uc):
    for M, E in [([1, 2], [0.0, 1.0]), ([1, 1, 2], [0.0, 1.0, 2.0]), ([0, 1, 2], [1.0, 2.0, 3.0]),
                 ([1, 2, 3], [1.0, np.inf, 3.0])]:
        with pytest.raises(uc.UCCSDError):
            uc.trotter_extrapolate(M, E)


def _dense_from_terms(x, z, c, nq):
    N = 1 << nq
    M = np.zeros((N, N))
    ys = np.arange(N, dtype=np.int64)
    for xi, zi, ci in zip(x.tolist(), z.tolist(), c.tolist()):
        sign = 1.0 - 2.0 * (np.array([bin(int(v) & zi).count("1") & 1 for v in ys]))
        M[ys ^ xi, ys] += ci * sign
    return M


@pytest.mark.parametrize("name,na,nb", [("8q", 2, 2), ("8q", 2, 1), ("12q", 3, 3)])
def test_scbk_tapered_spectrum_equals_the_parity_sector(uc, oracle_mod, name, na, nb):
    # the tapered (n - 2)-qubit Hamiltonian has exactly the eigenvalues of H on
    # the states with the alpha and total electron parities of (na, na + nb)
    w = synth.workload(name)
    n_orb = w["n_orb"]
    n = 2 * n_orb
    x, z, c, nq = uc.pauli_terms_scbk(n_orb, w["h"], w["eri"], 0.0, na, nb)
    assert nq == n - 2
    T = _dense_from_terms(x, z, c, nq)
    assert np.allclose(T, T.T, atol=1e-12)
    amask = sum(1 << q for q in range(0, n, 2))
    states = [s for s in range(1 << n)
              if bin(s & amask).count("1") % 2 == na % 2 and bin(s).count("1") % 2 == (na + nb) % 2]
    Hs = np.zeros((len(states), len(states)))
    pos = {s: i for i, s in enumerate(states)}
    for i, s in enumerate(states):
        e = np.zeros(1 << n, dtype=np.complex128)
        e[s] = 1.0
        col = oracle_mod.h_apply(n_orb, w["h"], w["eri"], 0.0, e).real
        for t_ in np.nonzero(col)[0]:
            Hs[pos[int(t_)], i] = col[t_]
    ev_t = np.linalg.eigvalsh(T)
    ev_h = np.linalg.eigvalsh(Hs)
    assert np.max(np.abs(ev_t - ev_h)) < 1e-9
    # the sector ground state (FCI of the paper's CAS-CI) is among them
    e_fci = oracle_mod.fci_energy(n_orb, w["h"], w["eri"], 0.0, na, nb)
    assert np.min(np.abs(ev_t - e_fci)) < 1e-9


def test_scbk_rejects_bad_input(uc):
    w = synth.workload("8q")
    with pytest.raises(uc.UCCSDError):
        uc.pauli_terms_scbk(1, w["h"][:1, :1], w["eri"][:1, :1, :1, :1], 0.0, 1, 1)
    with pytest.raises(uc.UCCSDError):
        uc.pauli_terms_scbk(4, w["h"], w["eri"], 0.0, 5, 2)
