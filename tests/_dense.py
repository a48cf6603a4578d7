"""Independent dense Jordan-Wigner construction used to pin the oracle.

Ladder operators are built as Kronecker products of 2x2 matrices (qubit q is
bit q of the basis index, so qubit n-1 is the leftmost Kronecker factor):
    a_q = I x ... x I x s x Z x ... x Z,   s = |0><1|,  Z = diag(1, -1)
with Z on the qubits below q.  Nothing here shares code with the oracle's
bit-string ladder arithmetic.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

_I = sp.identity(2, format="csr", dtype=np.float64)
_Z = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, -1.0]]))
_S = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |0><1|


@functools.lru_cache(maxsize=None)
def ann(n: int, q: int):
    op = None
    for site in range(n - 1, -1, -1):
        m = _I if site > q else (_S if site == q else _Z)
        op = m if op is None else sp.kron(op, m, format="csr")
    return op.tocsr()


def cre(n: int, q: int):
    return ann(n, q).T.tocsr()


def hamiltonian(n_orb, h, eri, e_core=0.0):
    """Eq. 2 with g_PQRS = (pr|qs) delta(s_P,s_R) delta(s_Q,s_S)."""
    n = 2 * n_orb
    N = 1 << n
    H = sp.identity(N, format="csr") * e_core
    for P in range(n):
        for Q in range(n):
            if P % 2 != Q % 2:
                continue
            c = h[P // 2, Q // 2]
            if c != 0.0:
                H = H + c * (cre(n, P) @ ann(n, Q))
    for P in range(n):
        for Q in range(n):
            for R in range(n):
                if P % 2 != R % 2:
                    continue
                for S in range(n):
                    if Q % 2 != S % 2:
                        continue
                    g = eri[P // 2, R // 2, Q // 2, S // 2]
                    if g != 0.0:
                        H = H + 0.5 * g * (cre(n, P) @ cre(n, Q) @ ann(n, S) @ ann(n, R))
    return H.tocsr()


def generator(n, ex):
    i, j, a, b = (int(v) for v in ex)
    if j < 0:
        tau = cre(n, a) @ ann(n, i)
    else:
        tau = cre(n, a) @ cre(n, b) @ ann(n, j) @ ann(n, i)
    return (tau - tau.T).toarray()


def number_op(n):
    N = 1 << n
    return np.array([bin(x).count("1") for x in range(N)], dtype=float)


def sz_op(n):
    N = 1 << n
    amask = sum(1 << q for q in range(0, n, 2))
    return np.array([0.5 * (bin(x & amask).count("1") - bin(x & ~amask & (N - 1)).count("1"))
                     for x in range(N)])


# Pauli matrices for the Pauli-string expansion pin.
PAULI = {
    "I": np.eye(2),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def pauli_string(labels):
    """labels[q] for qubit q; qubit n-1 is the leftmost Kronecker factor."""
    op = np.array([[1.0 + 0j]])
    for q in range(len(labels) - 1, -1, -1):
        op = np.kron(op, PAULI[labels[q]])
    return op
