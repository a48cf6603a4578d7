"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds random-number generation and input construction only; it
contains none of the method's arithmetic (no Hamiltonian action, no ansatz, no
energy).  Both the CPU oracle and the CUDA path consume exactly the arrays it
returns, so the two sides see identical bytes.

Generators (published definitions, restated):
  * splitmix64 (S. Vigna) seeds the state of
  * xoshiro256** (D. Blackman and S. Vigna, 2018).
  * uniform u = (r >> 11) * 2**-53 in [0, 1).
  * standard normals by the Box-Muller transform, consumed in pairs: the
    second value of a pair is cached and returned by the next draw.

Integral recipe (synthetic stand-in for the FMO fragment integrals of the
paper, Section 2.2, which are not available):
  (i)   h_pq for p < q in row-major order ~ N(0, 1), mirrored to q > p; the
        diagonal is replaced by linspace(-2, -0.5, n_orb) ascending, so the
        lowest orbitals are the occupied ones of the reference determinant.
  (ii)  Cholesky-like vectors L^k_pq for k = 0..n_chol-1 and p <= q row-major
        ~ N(0, 1) / sqrt(n_chol), mirrored.
  (iii) (pq|rs) = sum_k L^k_pq L^k_rs: chemist-notation integrals with the
        8-fold permutational symmetry of real orbitals, positive semidefinite
        as a (pq),(rs) matrix.
  e_core = 0.
Amplitude vectors theta use a separate generator stream.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class SplitMix64:
    """splitmix64 (Vigna): a 64-bit counter with an avalanche output mix."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


class Xoshiro256StarStar:
    """xoshiro256** (Blackman and Vigna), state filled from splitmix64(seed)."""

    def __init__(self, seed: int):
        sm = SplitMix64(seed)
        self.s = [sm.next() for _ in range(4)]
        self._spare = None

    def next(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (2.0 ** -53)

    def normal(self) -> float:
        """Standard normal by Box-Muller; pairs are consumed, spare cached."""
        if self._spare is not None:
            v, self._spare = self._spare, None
            return v
        # u1 in (0, 1] so that log(u1) is finite.
        u1 = ((self.next() >> 11) + 1) * (2.0 ** -53)
        u2 = (self.next() >> 11) * (2.0 ** -53)
        r = math.sqrt(-2.0 * math.log(u1))
        z0 = r * math.cos(2.0 * math.pi * u2)
        z1 = r * math.sin(2.0 * math.pi * u2)
        self._spare = z1
        return z0


def make_integrals(n_orb: int, n_chol: int, seed: int, offdiag: float = 1.0,
                   chol: float = 1.0):
    """Synthetic one- and two-electron integrals (recipe in the module doc).

    offdiag and chol scale the off-diagonal h_pq and the Cholesky-like
    vectors (1.0: the recipe above; smaller values give weakly correlated
    fragments dominated by their reference determinant).
    Returns (h, eri, e_core): h is (n_orb, n_orb) float64 symmetric,
    eri is (n_orb,)*4 float64 chemist-notation (pq|rs), e_core = 0.0.
    """
    rng = Xoshiro256StarStar(seed)
    h = np.zeros((n_orb, n_orb), dtype=np.float64)
    for p in range(n_orb):
        for q in range(p + 1, n_orb):
            v = rng.normal() * offdiag
            h[p, q] = v
            h[q, p] = v
    diag = np.linspace(-2.0, -0.5, n_orb) if n_orb > 1 else np.array([-2.0])
    for p in range(n_orb):
        h[p, p] = diag[p]
    L = np.zeros((n_chol, n_orb, n_orb), dtype=np.float64)
    scale = chol / math.sqrt(n_chol)
    for k in range(n_chol):
        for p in range(n_orb):
            for q in range(p, n_orb):
                v = rng.normal() * scale
                L[k, p, q] = v
                L[k, q, p] = v
    Lm = L.reshape(n_chol, n_orb * n_orb)
    eri = (Lm.T @ Lm).reshape(n_orb, n_orb, n_orb, n_orb)
    # Enforce exact 8-fold symmetry against matmul rounding order.
    eri = 0.5 * (eri + eri.transpose(2, 3, 0, 1))
    eri = 0.5 * (eri + eri.transpose(1, 0, 2, 3))
    eri = 0.5 * (eri + eri.transpose(0, 1, 3, 2))
    return np.ascontiguousarray(h), np.ascontiguousarray(eri), 0.0


def theta_uniform(K: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = Xoshiro256StarStar(seed)
    return np.array([lo + (hi - lo) * rng.uniform() for _ in range(K)],
                    dtype=np.float64)


def theta_normal(K: int, std: float, seed: int) -> np.ndarray:
    rng = Xoshiro256StarStar(seed)
    return np.array([std * rng.normal() for _ in range(K)], dtype=np.float64)


def random_state(n_qubits: int, seed: int, sector=None) -> np.ndarray:
    """Random normalised complex vector (test input), optionally supported
    only on the basis states accepted by ``sector`` (a callable x -> bool)."""
    rng = Xoshiro256StarStar(seed)
    N = 1 << n_qubits
    v = np.zeros(N, dtype=np.complex128)
    for x in range(N):
        if sector is None or sector(x):
            re = rng.normal()
            im = rng.normal()
            v[x] = complex(re, im)
    nrm = np.linalg.norm(v)
    return v / nrm if nrm > 0 else v


# Workloads with the shapes of the paper's fragments (monomers 8-12 qubits,
# dimers 16-18 qubits) plus a 26-qubit scale-up.  n_qubits = 2 * n_orb under
# the Jordan-Wigner mapping; closed shell n_alpha = n_beta = n_elec / 2.
WORKLOADS = {
    "8q": dict(n_orb=4, n_elec=4, n_chol=6, seed=0),
    "12q": dict(n_orb=6, n_elec=6, n_chol=10, seed=1),
    "18q": dict(n_orb=9, n_elec=10, n_chol=16, seed=2),
    "26q": dict(n_orb=13, n_elec=12, n_chol=20, seed=4),
}


def workload(name: str):
    w = WORKLOADS[name]
    h, eri, e_core = make_integrals(w["n_orb"], w["n_chol"], w["seed"])
    return dict(w, h=h, eri=eri, e_core=e_core,
                n_alpha=w["n_elec"] // 2, n_beta=w["n_elec"] // 2)


def non_interacting_dimer(h_a, eri_a, n_occ_a, h_b, eri_b, n_occ_b):
    """Integrals of two fragments with no integral between them (a dimer at
    infinite separation, the size-consistency setting of the paper's
    Section 3.2) in localised orbitals, ordered [A occupied, B occupied,
    A virtual, B virtual] so that the lowest orbitals form the product
    reference determinant.  Returns (h, eri, perm) with perm[new] = old index
    in the block-diagonal order [A orbitals, B orbitals]."""
    na, nb = h_a.shape[0], h_b.shape[0]
    n = na + nb
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    h[:na, :na] = h_a
    h[na:, na:] = h_b
    eri[:na, :na, :na, :na] = eri_a
    eri[na:, na:, na:, na:] = eri_b
    perm = (list(range(n_occ_a)) + [na + i for i in range(n_occ_b)] +
            list(range(n_occ_a, na)) + [na + i for i in range(n_occ_b, nb)])
    perm = np.array(perm)
    h = h[np.ix_(perm, perm)]
    eri = eri[np.ix_(perm, perm, perm, perm)]
    return np.ascontiguousarray(h), np.ascontiguousarray(eri), perm


def rotate_orbitals(h, eri, U):
    """Integrals in the rotated orbitals phi'_p = sum_q U[q, p] phi_q
    (U orthogonal): h' = U^T h U, (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd)."""
    h2 = U.T @ h @ U
    e2 = np.einsum("abcd,ap,bq,cr,ds->pqrs", eri, U, U, U, U, optimize=True)
    # restore exact 8-fold symmetry against summation-order rounding
    e2 = 0.5 * (e2 + e2.transpose(2, 3, 0, 1))
    e2 = 0.5 * (e2 + e2.transpose(1, 0, 2, 3))
    e2 = 0.5 * (e2 + e2.transpose(0, 1, 3, 2))
    return np.ascontiguousarray(0.5 * (h2 + h2.T)), np.ascontiguousarray(e2)


def pair_mixing(n_occ, n_virt, angle=math.pi / 4):
    """Orthogonal U for a dimer ordered [A occ, B occ, A virt, B virt] with
    n_occ occupied and n_virt virtual orbitals per fragment: orbital i of A
    and orbital i of B (occupied with occupied, virtual with virtual) are
    rotated into each other by `angle`.  At pi/4 these are the
    symmetric/antisymmetric combinations, the canonical orbitals of two
    identical non-interacting fragments (delocalised over the dimer)."""
    n = 2 * (n_occ + n_virt)
    U = np.eye(n)
    c, s = math.cos(angle), math.sin(angle)
    pairs = [(i, n_occ + i) for i in range(n_occ)]
    pairs += [(2 * n_occ + a, 2 * n_occ + n_virt + a) for a in range(n_virt)]
    for p, q in pairs:
        U[p, p], U[q, p] = c, s
        U[p, q], U[q, q] = -s, c
    return U


def fmo_trimer(seed: int, coupling: float, n_frag: int = 3, n_orb_frag: int = 4,
               n_occ_frag: int = 2, n_chol_frag: int = 5, n_chol_cross: int = 4):
    """Integrals of a synthetic supersystem of n_frag fragments (the FMO
    setting of the paper's Section 2.1), each with n_orb_frag localised
    orbitals of which the n_occ_frag lowest are occupied.

    Orbital order: fragment after fragment, occupied before virtual within a
    fragment.  Draw order (one generator, seed):
      (i)   for each fragment: h_pq (p < q within the fragment) ~ N(0, 1),
            diagonal linspace(-2, -0.5, n_orb_frag);
      (ii)  for each pair of orbitals of different fragments (p < q,
            row-major): h_pq ~ N(0, 1) * coupling;
      (iii) for each fragment, n_chol_frag vectors L_pq (p <= q within the
            fragment) ~ N(0, 1) / sqrt(n_chol_frag);
      (iv)  n_chol_cross vectors on all pairs p <= q ~ N(0, 1) /
            sqrt(n_chol_cross) * coupling;
      (pq|rs) = sum over all vectors of L_pq L_rs (8-fold symmetric, PSD).
    coupling = 0 gives non-interacting fragments (block-diagonal integrals).
    Returns dict(h, eri, frag_orbs, frag_nocc)."""
    rng = Xoshiro256StarStar(seed)
    n = n_frag * n_orb_frag
    frag_orbs = [list(range(f * n_orb_frag, (f + 1) * n_orb_frag)) for f in range(n_frag)]
    frag_of = [p // n_orb_frag for p in range(n)]
    h = np.zeros((n, n))
    for orbs in frag_orbs:
        for a, p in enumerate(orbs):
            for q in orbs[a + 1:]:
                h[p, q] = h[q, p] = rng.normal()
        for a, p in enumerate(orbs):
            h[p, p] = -2.0 + 1.5 * a / max(1, n_orb_frag - 1)
    for p in range(n):
        for q in range(p + 1, n):
            if frag_of[p] != frag_of[q]:
                h[p, q] = h[q, p] = rng.normal() * coupling
    vecs = []
    for orbs in frag_orbs:
        for _ in range(n_chol_frag):
            L = np.zeros((n, n))
            for a, p in enumerate(orbs):
                for q in orbs[a:]:
                    L[p, q] = L[q, p] = rng.normal() / math.sqrt(n_chol_frag)
            vecs.append(L)
    for _ in range(n_chol_cross):
        L = np.zeros((n, n))
        for p in range(n):
            for q in range(p, n):
                L[p, q] = L[q, p] = rng.normal() / math.sqrt(n_chol_cross) * coupling
        vecs.append(L)
    eri = np.zeros((n, n, n, n))
    for L in vecs:
        eri += np.einsum("pq,rs->pqrs", L, L)
    return dict(h=h, eri=eri, frag_orbs=frag_orbs, frag_nocc=[n_occ_frag] * n_frag)


def stream_fragments(n_req: int, seed: int = 7):
    """stream_requests() with each fragment's integrals attached
    (h, eri, e_core, n_alpha, n_beta)."""
    out = []
    for d in stream_requests(n_req, seed):
        h, eri, e_core = make_integrals(d["n_orb"], d["n_chol"], d["seed"])
        out.append(dict(d, h=h, eri=eri, e_core=e_core, n_alpha=d["n_elec"] // 2,
                        n_beta=d["n_elec"] - d["n_elec"] // 2))
    return out


def stream_requests(n_req: int, seed: int = 7):
    """Fragment request mix of a two-body FMO job: 60% monomers with
    n_orb in {4,5,6} (8/10/12 qubits; 4/4/6 electrons) and 40% dimers with
    n_orb in {8,9} (16/18 qubits; 8/10 electrons).  Fragment r draws its
    integrals from seed 10000 + r with n_chol = n_orb + 1.  Inter-arrival
    gaps are unit-rate exponentials (scale them by 1/rate)."""
    rng = Xoshiro256StarStar(seed)
    out = []
    t = 0.0
    for r in range(n_req):
        t += -math.log(1.0 - rng.uniform())
        if rng.uniform() < 0.6:
            n_orb = (4, 5, 6)[min(2, int(3 * rng.uniform()))]
            n_elec = {4: 4, 5: 4, 6: 6}[n_orb]
        else:
            n_orb = (8, 9)[min(1, int(2 * rng.uniform()))]
            n_elec = {8: 8, 9: 10}[n_orb]
        out.append(dict(r=r, t_unit=t, n_orb=n_orb, n_elec=n_elec,
                        n_chol=n_orb + 1, seed=10000 + r))
    return out
