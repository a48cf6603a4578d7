"""UCCSD oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU restatement of the VQE-UCCSD correlation step of
arXiv:2402.17993 (Sections 2.2-2.3, Eqs. 2-6), used to check the CUDA
library.  Only the test suite, ``__graft_entry__.smoke`` and the benchmark's
CPU-baseline / reference leg may import this package.  It shares no code with
the CUDA path (``paper_2402_17993_gb300``) and never imports it.

The arithmetic lives in ``uccsd_oracle.c`` (ladder operators on occupation
bit strings; Eq. 2 literally and by Slater-Condon rules; Eq. 4 generators;
Eq. 5/6 schedules; adjoint gradient).  This module adds the list builders,
the dense-matrix helpers (FCI by numpy.linalg.eigh, Trotter-free energies by
scipy.linalg.expm on the full space and by scipy.sparse.linalg.expm_multiply
on the electron sector), the magnitude ordering of Section 2.3 with first-order
amplitudes, the Trotter-error extrapolation of Section 3.2, the FMO two-body
assembly of Section 2.1 (Eq. 1, embedded fragment integrals) and ctypes
marshalling.

Parity pins: every function here is checked against something other than
itself in ``tests/test_oracle_pins.py``, ``tests/test_oracle_trotter.py`` and
``tests/test_oracle_fmo.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "uccsd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        lib.oracle_h_apply_eq2.argtypes = [c_int, dp, dp, c_double, dp, dp]
        lib.oracle_h_apply_sc.argtypes = [c_int, dp, dp, c_double, dp, dp]
        lib.oracle_apply_generator.argtypes = [c_int, ip, dp, dp]
        lib.oracle_rotate.argtypes = [c_int, ip, c_double, dp]
        lib.oracle_energy_grad.argtypes = [c_int, dp, dp, c_double, c_int, c_int, c_int, ip,
                                           c_int, ip, dp, dp, c_int, c_int,
                                           dp, dp, dp, dp]
        lib.oracle_sector_size.argtypes = [c_int, c_int, c_int, ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_num_threads.restype = c_int
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_generator_sum_sector.argtypes = [c_int, c_int, c_int, c_int, ip, dp,
                                                    ctypes.c_int64, i64p, i64p, dp, i64p]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _cvec(psi: np.ndarray) -> np.ndarray:
    """complex128 vector -> contiguous interleaved float64 view."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return psi.view(np.float64)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------------------
# Lists (Eq. 4, Eq. 5, Eq. 6)
# ---------------------------------------------------------------------------
def hf_index(n_alpha: int, n_beta: int) -> int:
    """Reference determinant: lowest n_alpha alpha (even qubits) and n_beta
    beta (odd qubits) spin orbitals occupied."""
    x = 0
    for p in range(n_alpha):
        x |= 1 << (2 * p)
    for p in range(n_beta):
        x |= 1 << (2 * p + 1)
    return x


def excitations(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Spin-conserving UCCSD excitation list of Eq. 4 over spin orbitals.

    Singles (i, a): i occupied, a virtual in |HF>, same spin.  Doubles
    (i < j, a < b): i, j occupied, a, b virtual, spin multiset conserved.
    Singles first, then doubles, each in lexicographic order of the tuple.
    Rows are (i, j, a, b) with j = b = -1 for singles.
    """
    n = 2 * n_orb
    hf = hf_index(n_alpha, n_beta)
    occ = [p for p in range(n) if (hf >> p) & 1]
    vir = [p for p in range(n) if not (hf >> p) & 1]
    rows = []
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                rows.append((i, -1, a, -1))
    for i in occ:
        for j in occ:
            if j <= i:
                continue
            for a in vir:
                for b in vir:
                    if b <= a:
                        continue
                    if sorted((i % 2, j % 2)) == sorted((a % 2, b % 2)):
                        rows.append((i, j, a, b))
    return np.array(rows, dtype=np.int32).reshape(-1, 4)


def schedule(K: int, order: int = 1, M: int = 1):
    """Trotter schedule as (op_k, op_scale) in acting order.

    order 1 (Eq. 5): [exp(theta_1 G_1/M) ... exp(theta_K G_K/M)]^M with
    excitation 1 acting first.  order 2 (Eq. 6): each of the M repetitions
    is the list 1..K then K..1, every factor with theta/(2M).
    """
    ks, sc = [], []
    for _ in range(M):
        if order == 1:
            ks += list(range(K))
            sc += [1.0 / M] * K
        elif order == 2:
            ks += list(range(K)) + list(range(K - 1, -1, -1))
            sc += [1.0 / (2 * M)] * (2 * K)
        else:
            raise ValueError("order must be 1 or 2")
    return np.array(ks, dtype=np.int32), np.array(sc, dtype=np.float64)


# ---------------------------------------------------------------------------
# Operator actions
# ---------------------------------------------------------------------------
def h_apply(n_orb, h, eri, e_core, psi, method="sc"):
    """sigma = H psi (+ e_core psi) by Eq. 2 literally ('eq2') or by
    Slater-Condon rules ('sc')."""
    lib = _load()
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    p = _cvec(psi)
    out = np.zeros_like(p)
    fn = lib.oracle_h_apply_eq2 if method == "eq2" else lib.oracle_h_apply_sc
    _check(fn(n_orb, _dp(h), _dp(eri), float(e_core), _dp(p), _dp(out)), "h_apply")
    return out.view(np.complex128)


def apply_generator(n_qubits, ex, psi):
    """G psi for one excitation row (i, j, a, b) (Eq. 4, G = tau - tau^dag)."""
    lib = _load()
    ex = np.ascontiguousarray(ex, dtype=np.int32)
    p = _cvec(psi)
    out = np.zeros_like(p)
    _check(lib.oracle_apply_generator(n_qubits, _ip(ex), _dp(p), _dp(out)), "apply_generator")
    return out.view(np.complex128)


def rotate(n_qubits, ex, phi, psi):
    """exp(phi G) psi for one excitation."""
    lib = _load()
    ex = np.ascontiguousarray(ex, dtype=np.int32)
    p = _cvec(np.array(psi, dtype=np.complex128, copy=True)).copy()
    _check(lib.oracle_rotate(n_qubits, _ip(ex), float(phi), _dp(p)), "rotate")
    return p.view(np.complex128)


def energy_grad(n_orb, h, eri, e_core, n_alpha, n_beta, ijab, theta,
                order=1, M=1, op_k=None, op_scale=None, grad=True,
                sector=False, method="sc", want_state=False):
    """Trotterised UCCSD energy (and adjoint gradient) for one theta.

    Returns (E, g or None[, psi, sigma]).
    """
    lib = _load()
    n = 2 * n_orb
    ijab = np.ascontiguousarray(ijab, dtype=np.int32).reshape(-1, 4)
    K = ijab.shape[0]
    theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(K)
    if op_k is None:
        op_k, op_scale = schedule(K, order, M)
    op_k = np.ascontiguousarray(op_k, dtype=np.int32)
    op_scale = np.ascontiguousarray(op_scale, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    E = np.zeros(1)
    g = np.zeros(max(K, 1))
    null = ctypes.POINTER(ctypes.c_double)()
    psi = sig = None
    if want_state:
        psi = np.zeros(2 << n)
        sig = np.zeros(2 << n)
    rc = lib.oracle_energy_grad(n_orb, _dp(h), _dp(eri), float(e_core), n_alpha, n_beta,
                                K, _ip(ijab), len(op_k), _ip(op_k), _dp(op_scale),
                                _dp(theta), 1 if sector else 0, 0 if method == "eq2" else 1,
                                _dp(E), _dp(g) if grad else null,
                                _dp(psi) if want_state else null,
                                _dp(sig) if want_state else null)
    _check(rc, "energy_grad")
    out = (float(E[0]), g[:K].copy() if grad else None)
    if want_state:
        out = out + (psi.view(np.complex128), sig.view(np.complex128))
    return out


# ---------------------------------------------------------------------------
# Dense helpers (small cases only)
# ---------------------------------------------------------------------------
def sector_basis(n_qubits, n_alpha, n_beta):
    amask = sum(1 << q for q in range(0, n_qubits, 2))
    return np.array([x for x in range(1 << n_qubits)
                     if bin(x & amask).count("1") == n_alpha
                     and bin(x & ~amask).count("1") == n_beta], dtype=np.int64)


def sector_size(n_qubits, n_alpha, n_beta) -> int:
    c = ctypes.c_int64(0)
    _check(_load().oracle_sector_size(n_qubits, n_alpha, n_beta, ctypes.byref(c)), "sector_size")
    return int(c.value)


def h_sector_matrix(n_orb, h, eri, e_core, n_alpha, n_beta, method="sc"):
    """Dense H restricted to the (n_alpha, n_beta) sector, column by column."""
    n = 2 * n_orb
    basis = sector_basis(n, n_alpha, n_beta)
    D = len(basis)
    Hs = np.zeros((D, D))
    e = np.zeros(1 << n, dtype=np.complex128)
    for c, x in enumerate(basis):
        e[:] = 0
        e[x] = 1.0
        col = h_apply(n_orb, h, eri, e_core, e, method)
        Hs[:, c] = col[basis].real
    return Hs, basis


def fci_energy(n_orb, h, eri, e_core, n_alpha, n_beta, method="sc"):
    """Exact ground-state energy in the sector (CAS-CI of the paper's
    Section 2.3) by numpy.linalg.eigh."""
    Hs, _ = h_sector_matrix(n_orb, h, eri, e_core, n_alpha, n_beta, method)
    return float(np.linalg.eigvalsh(Hs)[0])


def generator_matrix(n_qubits, ex):
    """Dense 2^n x 2^n matrix of G for one excitation (small n only)."""
    N = 1 << n_qubits
    Gm = np.zeros((N, N))
    e = np.zeros(N, dtype=np.complex128)
    for x in range(N):
        e[:] = 0
        e[x] = 1.0
        Gm[:, x] = apply_generator(n_qubits, ex, e).real
    return Gm


def trotter_free_energy(n_orb, h, eri, e_core, n_alpha, n_beta, ijab, theta):
    """E of exp(sum_k theta_k G_k)|HF> (no Trotterisation) by dense
    scipy.linalg.expm, as the paper's expm_multiply reference (Sec. 3.2)."""
    import scipy.linalg
    n = 2 * n_orb
    A = np.zeros((1 << n, 1 << n))
    for k, ex in enumerate(np.asarray(ijab).reshape(-1, 4)):
        A += theta[k] * generator_matrix(n, ex)
    hf = np.zeros(1 << n, dtype=np.complex128)
    hf[hf_index(n_alpha, n_beta)] = 1.0
    psi = scipy.linalg.expm(A) @ hf
    sig = h_apply(n_orb, h, eri, e_core, psi)
    return float(np.vdot(psi, sig).real), psi


# ---------------------------------------------------------------------------
# Trotter-product ordering (Section 2.3) and Trotter-error extrapolation
# (Section 3.2, Fig. 3)
# ---------------------------------------------------------------------------
def fock_diagonal(n_orb, h, eri, n_alpha, n_beta):
    """Spin-orbital Fock diagonal of the reference determinant,
    eps_P = h_pp + sum_{I occupied} [(pp|ii) - delta(s_P, s_I) (pi|ip)],
    for spin orbital P = 2p + s_P (the orbital energies of Moller-Plesset
    partitioning)."""
    n = 2 * n_orb
    hf = hf_index(n_alpha, n_beta)
    eps = np.zeros(n)
    for P in range(n):
        p = P >> 1
        v = h[p, p]
        for I in range(n):
            if not (hf >> I) & 1:
                continue
            i = I >> 1
            v += eri[p, p, i, i]
            if (P & 1) == (I & 1):
                v -= eri[p, i, i, p]
        eps[P] = v
    return eps


def mp1_amplitudes(n_orb, h, eri, e_core, n_alpha, n_beta, ijab):
    """First-order (Moller-Plesset) amplitude of every excitation,
    t_k = <Phi_k|H|HF> / (eps_i + eps_j - eps_a - eps_b), Phi_k = tau_k|HF>
    (singles: eps_i - eps_a).  The numerator is taken from the state vector:
    tau_k|HF> = G_k|HF> because tau_k^dag annihilates |HF>.
    Returns (t, numerators)."""
    n = 2 * n_orb
    hf = np.zeros(1 << n, dtype=np.complex128)
    hf[hf_index(n_alpha, n_beta)] = 1.0
    sig = h_apply(n_orb, h, eri, e_core, hf)
    eps = fock_diagonal(n_orb, h, eri, n_alpha, n_beta)
    rows = np.asarray(ijab, dtype=np.int32).reshape(-1, 4)
    t = np.zeros(len(rows))
    num = np.zeros(len(rows))
    for k, (i, j, a, b) in enumerate(rows):
        phi = apply_generator(n, rows[k], hf)
        num[k] = np.vdot(phi, sig).real
        den = eps[i] - eps[a] + ((eps[j] - eps[b]) if j >= 0 else 0.0)
        t[k] = num[k] / den
    return t, num


def magnitude_order(ijab, t):
    """Magnitude ordering of the cluster operators (Section 2.3): rows by
    decreasing |t|, equal magnitudes in list order.  Returns (rows, perm)
    with rows = ijab[perm]."""
    rows = np.asarray(ijab, dtype=np.int32).reshape(-1, 4)
    mag = np.abs(np.asarray(t, dtype=np.float64))
    perm = sorted(range(len(rows)), key=lambda k: (-mag[k], k))
    perm = np.array(perm, dtype=np.int64)
    return rows[perm], perm


def trotter_extrapolate(Ms, Es):
    """Least-squares fit of E(M) = alpha (1/M)^beta + gamma (Section 3.2,
    Fig. 3) by scipy.optimize.curve_fit (Levenberg-Marquardt).
    Returns (alpha, beta, gamma); gamma estimates the Trotter-free energy."""
    import scipy.optimize
    x = 1.0 / np.asarray(Ms, dtype=np.float64)
    E = np.asarray(Es, dtype=np.float64)

    def model(x, a, b, g):
        return a * x ** b + g

    p0 = (E[0] - E[-1] if E[0] != E[-1] else 1.0, 2.0, E[-1])
    popt, _ = scipy.optimize.curve_fit(model, x, E, p0=p0, maxfev=100000,
                                       xtol=1e-15, ftol=1e-15, gtol=1e-15)
    return float(popt[0]), float(popt[1]), float(popt[2])


# ---------------------------------------------------------------------------
# Trotter-free ansatz exp(T - T^dag)|HF> (Eq. 3) on the electron sector
# ---------------------------------------------------------------------------
def generator_sum_sector(n_qubits, n_alpha, n_beta, ijab, theta):
    """A = sum_k theta_k G_k as a scipy.sparse CSC matrix on the sector basis
    (ascending basis states, the order of sector_basis), built column by
    column from the ladder operators."""
    import scipy.sparse
    lib = _load()
    ijab = np.ascontiguousarray(ijab, dtype=np.int32).reshape(-1, 4)
    theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(ijab.shape[0])
    dim = sector_size(n_qubits, n_alpha, n_beta)
    nnz = ctypes.c_int64(0)
    col = np.zeros(dim + 1, dtype=np.int64)
    i64p = ctypes.POINTER(ctypes.c_int64)
    _check(lib.oracle_generator_sum_sector(n_qubits, n_alpha, n_beta, ijab.shape[0], _ip(ijab),
                                           _dp(theta), 0, col.ctypes.data_as(i64p), None, None,
                                           ctypes.byref(nnz)), "generator_sum_sector")
    row = np.zeros(max(nnz.value, 1), dtype=np.int64)
    val = np.zeros(max(nnz.value, 1))
    _check(lib.oracle_generator_sum_sector(n_qubits, n_alpha, n_beta, ijab.shape[0], _ip(ijab),
                                           _dp(theta), nnz.value, col.ctypes.data_as(i64p),
                                           row.ctypes.data_as(i64p), _dp(val),
                                           ctypes.byref(nnz)), "generator_sum_sector")
    n = nnz.value
    return scipy.sparse.csc_matrix((val[:n], row[:n], col), shape=(dim, dim))


def trotter_free_energy_sector(n_orb, h, eri, e_core, n_alpha, n_beta, ijab, theta):
    """E of exp(sum_k theta_k G_k)|HF> on the sector by
    scipy.sparse.linalg.expm_multiply, the routine named for the paper's
    Trotter-free reference (Section 3.2); H acts by Slater-Condon rules.
    Returns (E, psi) with psi the full 2^n vector."""
    import scipy.sparse.linalg
    n = 2 * n_orb
    A = generator_sum_sector(n, n_alpha, n_beta, ijab, theta)
    basis = sector_basis(n, n_alpha, n_beta)
    e0 = np.zeros(len(basis))
    e0[int(np.searchsorted(basis, hf_index(n_alpha, n_beta)))] = 1.0
    v = scipy.sparse.linalg.expm_multiply(A, e0)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[basis] = v
    sig = h_apply(n_orb, h, eri, e_core, psi)
    return float(np.vdot(psi, sig).real), psi


def trotter_free_energy_grad_sector(n_orb, h, eri, e_core, n_alpha, n_beta, ijab, theta):
    """E and gradient of exp(A)|HF>, A = sum_k theta_k G_k, on the sector:
    dE/dtheta_k = 2 <H psi| L(A, G_k) |HF> with L the Frechet derivative of
    the matrix exponential (scipy.linalg.expm_frechet).  Dense sector
    matrices: small sectors only.  Returns (E, g)."""
    import scipy.linalg
    n = 2 * n_orb
    rows = np.asarray(ijab, dtype=np.int32).reshape(-1, 4)
    theta = np.asarray(theta, dtype=np.float64).reshape(len(rows))
    A = generator_sum_sector(n, n_alpha, n_beta, rows, theta).toarray()
    basis = sector_basis(n, n_alpha, n_beta)
    e0 = np.zeros(len(basis))
    e0[int(np.searchsorted(basis, hf_index(n_alpha, n_beta)))] = 1.0
    v = scipy.linalg.expm(A) @ e0
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[basis] = v
    sig = h_apply(n_orb, h, eri, e_core, psi)
    E = float(np.vdot(psi, sig).real)
    s = sig[basis].real
    g = np.zeros(len(rows))
    for k in range(len(rows)):
        Gk = generator_sum_sector(n, n_alpha, n_beta, rows[k:k + 1], [1.0]).toarray()
        L = scipy.linalg.expm_frechet(A, Gk, compute_expm=False)
        g[k] = 2.0 * s @ (L @ e0)
    return E, g


# ---------------------------------------------------------------------------
# FMO two-body assembly (Section 2.1, Eq. 1)
# ---------------------------------------------------------------------------
def fmo_fragment_integrals(h, eri, frag_orbs, frag_nocc, members):
    """Integrals of the fragment made of `members` (one monomer or two for a
    dimer) in the mean field of the other fragments' closed-shell reference
    determinants, written out element by element:
        h'_pq = h_pq + sum_{j in env occ} [2 (pq|jj) - (pj|jq)]
        (pq|rs)' = (pq|rs) restricted to the members' orbitals,
    orbitals ordered [members' occupied..., members' virtual...].
    Returns (h', eri', n_occ)."""
    occ, vir = [], []
    for f in members:
        occ += list(frag_orbs[f][:frag_nocc[f]])
        vir += list(frag_orbs[f][frag_nocc[f]:])
    sel = occ + vir
    env = []
    for f in range(len(frag_orbs)):
        if f not in members:
            env += list(frag_orbs[f][:frag_nocc[f]])
    m = len(sel)
    hp = np.zeros((m, m))
    for a, p in enumerate(sel):
        for b, q in enumerate(sel):
            v = h[p, q]
            for j in env:
                v += 2.0 * eri[p, q, j, j] - eri[p, j, j, q]
            hp[a, b] = v
    ep = np.zeros((m, m, m, m))
    for a, p in enumerate(sel):
        for b, q in enumerate(sel):
            for c, r in enumerate(sel):
                for d, s in enumerate(sel):
                    ep[a, b, c, d] = eri[p, q, r, s]
    return hp, ep, len(occ)


def fmo2_energy(E_monomer, E_dimer, n_frag):
    """Eq. 1: sum_{I<J} E_IJ - (N_f - 2) sum_I E_I, with E_monomer[I] and
    E_dimer[(I, J)] (I < J)."""
    total = 0.0
    for i in range(n_frag):
        for j in range(i + 1, n_frag):
            total += E_dimer[(i, j)]
    for i in range(n_frag):
        total -= (n_frag - 2) * E_monomer[i]
    return total
