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
