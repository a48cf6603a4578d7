"""Host check of the H-apply's split Jordan-Wigner signs.

The H-apply (kernels.cu) evaluates the parity popc(source & J) of a group's
interval mask J = XOR over its flipped qubits q of (bits below q), minus
the flipped bits, as a sum of terms that each depend on fewer indices
(alpha orbital i on qubit 2i, beta orbital j on qubit 2j + 1).  These tests
compare each split with the direct formula on random strings; a wrong
split (a dropped term, an off-by-one in a prefix) fails them.
"""
import random

import pytest


def interval_mask(x):
    m, v = 0, x
    while v:
        m ^= (v & -v) - 1
        v &= v - 1
    return m & ~x


def split_packed(J, n):
    ja = jb = 0
    for k in range(2 * n):
        if (J >> k) & 1:
            if k & 1:
                jb |= 1 << (k >> 1)
            else:
                ja |= 1 << (k >> 1)
    return ja, jb


def pc(v):
    return bin(v).count("1")


def prefix_parity(x):
    """Bit v = parity of bits 0..v (the kernel's shift-and-XOR ladder)."""
    x ^= x << 1
    x ^= x << 2
    x ^= x << 4
    x ^= x << 8
    return x & 0xFFFF


def direct(sa, yb, x, n):
    ja, jb = split_packed(interval_mask(x), n)
    return (pc(sa & ja) + pc(yb & jb)) & 1


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_group_sign_split(seed):
    rng = random.Random(seed)
    for _ in range(20000):
        n = rng.randint(2, 13)
        p, q = rng.sample(range(n), 2)
        j, b = rng.sample(range(n), 2)
        sR = (rng.getrandbits(n) | (1 << p)) & ~(1 << q)   # target row: p occupied
        sc = (rng.getrandbits(n) | (1 << j)) & ~(1 << b)   # target column: j occupied
        sa = sR ^ (1 << p) ^ (1 << q)
        yb = sc ^ (1 << j) ^ (1 << b)
        x = (1 << 2 * p) | (1 << 2 * q) | (1 << (2 * j + 1)) | (1 << (2 * b + 1))
        ja, _ = split_packed(interval_mask(x), n)
        apq = ((1 << p) - 1) ^ ((1 << q) - 1)
        lo, hi = min(j, b), max(j, b)
        between = ((1 << hi) - 1) & ~((2 << lo) - 1)
        table = (pc(sa & ja) ^ (apq >> j)) & 1           # staged table entry
        column = pc(sc & between) & 1                    # negated half (bmix)
        single = pc(sc & apq) & 1                        # flips the partial sum
        assert table ^ column ^ single == direct(sa, yb, x, n)


@pytest.mark.parametrize("seed", [3, 4])
def test_beta_single_and_double_sign_split(seed):
    rng = random.Random(seed)
    for _ in range(20000):
        n = rng.randint(4, 13)
        sR = rng.getrandbits(n)
        pa = prefix_parity(sR)
        # beta single j -> b on the own row
        j, b = rng.sample(range(n), 2)
        sc = (rng.getrandbits(n) | (1 << j)) & ~(1 << b)
        pab = pa ^ prefix_parity(sc << 1)
        lo, hi = min(j, b), max(j, b)
        row = ((pa >> lo) ^ (pa >> hi)) & 1
        col = (pc(sc & ((1 << j) - 1)) + pc(sc & ((1 << b) - 1)) + (b > j)) & 1
        assert row ^ col == direct(sR, sc ^ (1 << j) ^ (1 << b), (1 << (2 * j + 1)) | (1 << (2 * b + 1)), n)
        assert row ^ col == ((pab >> j) ^ (pab >> b) ^ (b > j)) & 1
        # beta double j1 j2 -> b1 b2
        j1, j2, b1, b2 = rng.sample(range(n), 4)
        j1, j2 = min(j1, j2), max(j1, j2)
        b1, b2 = min(b1, b2), max(b1, b2)
        sc = (rng.getrandbits(n) | (1 << j1) | (1 << j2)) & ~((1 << b1) | (1 << b2))
        pab = pa ^ prefix_parity(sc << 1)
        M = ((1 << j1) - 1) ^ ((1 << j2) - 1) ^ ((1 << b1) - 1) ^ ((1 << b2) - 1)
        own = ((M >> j1) ^ (M >> j2)) & 1                # folded into the table
        lane = ((pab >> j1) ^ (pab >> j2) ^ (pab >> b1) ^ (pab >> b2)) & 1
        x = sum(1 << (2 * v + 1) for v in (j1, j2, b1, b2))
        yb = sc ^ (1 << j1) ^ (1 << j2) ^ (1 << b1) ^ (1 << b2)
        assert own ^ lane == direct(sR, yb, x, n)


def test_diagonal_row_column_split():
    """The diagonal's occupation form over all occupied qubits equals the
    row part + column part + alpha-beta pair sums per beta orbital."""
    rng = random.Random(5)
    for _ in range(200):
        n_orb = rng.randint(2, 9)
        nq = 2 * n_orb
        qa = [rng.randint(-1000, 1000) for _ in range(nq)]
        qb = [[rng.randint(-1000, 1000) if r > q else 0 for r in range(nq)] for q in range(nq)]
        sR, sc = rng.getrandbits(n_orb), rng.getrandbits(n_orb)
        occ = [2 * i for i in range(n_orb) if sR >> i & 1] + [2 * j + 1 for j in range(n_orb) if sc >> j & 1]
        occ.sort()
        full = sum(qa[a] for a in occ) + sum(qb[a][r] for k, a in enumerate(occ) for r in occ[k + 1:])
        A = [2 * i for i in range(n_orb) if sR >> i & 1]
        B = [2 * j + 1 for j in range(n_orb) if sc >> j & 1]
        rowpart = sum(qa[a] for a in A) + sum(qb[a][a2] for k, a in enumerate(A) for a2 in A[k + 1:])
        colpart = sum(qa[r] for r in B) + sum(qb[r][r2] for k, r in enumerate(B) for r2 in B[k + 1:])
        xrow = {r: sum(qb[min(a, r)][max(a, r)] for a in A) for r in B}
        assert rowpart + colpart + sum(xrow.values()) == full
