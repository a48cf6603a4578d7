// Symmetry-conserving Bravyi-Kitaev qubit reduction of the Hamiltonian of
// Eq. 2 (the SCBKT encoding named in Section 2.3), host only.
//
// 1. Spin orbitals in up-then-down order: alpha orbital p on qubit p, beta
//    orbital p on qubit n/2 + p; Jordan-Wigner terms X^x Z^z in that order.
// 2. Bravyi-Kitaev tree by recursive halving of [0, n): qubit j of the
//    encoded basis holds the occupation parity of j and its descendants, so
//    b = B n over GF(2).  Node n/2 - 1 spans the alpha orbitals and the root
//    n - 1 spans all orbitals.
// 3. A Pauli term maps as X^x Z^z -> X^{B x} Z^{B^-T z} with the same real
//    coefficient (|n> -> |B n>; the phase (-1)^{z.n} = (-1)^{(B^-T z).b}).
// 4. H conserves N_alpha and N, so no term flips qubits n/2 - 1 and n - 1;
//    their Z operators are replaced by (-1)^{N_alpha} and (-1)^{N} and the two
//    qubits are removed, leaving n - 2 qubits.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "../../include/uccsd.h"
#include "jw.hpp"

namespace {

inline int popc(uint32_t v) { return __builtin_popcount(v); }

// rows[j] = orbitals whose occupations qubit j of the tree encoding sums.
std::vector<uint32_t> bk_tree_rows(int n) {
    std::vector<int> parent(n, -1);
    struct Rec {
        static void split(int l, int r, int par, std::vector<int> &parent) {
            if (l >= r) return;
            const int pivot = (l + r) >> 1;
            parent[pivot] = par;
            split(l, pivot, pivot, parent);
            split(pivot + 1, r, par, parent);
        }
    };
    Rec::split(0, n - 1, n - 1, parent);
    std::vector<uint32_t> rows(n, 0u);
    for (int j = 0; j < n; ++j)
        for (int a = j; a >= 0; a = parent[a]) rows[a] |= 1u << j;
    return rows;
}

// Inverse of an n x n GF(2) matrix given by rows (bit i of rows[r] = entry (r, i)).
bool gf2_inverse(std::vector<uint32_t> a, std::vector<uint32_t> *inv) {
    const int n = int(a.size());
    std::vector<uint32_t> e(n);
    for (int i = 0; i < n; ++i) e[i] = 1u << i;
    for (int c = 0; c < n; ++c) {
        int piv = -1;
        for (int r = c; r < n; ++r)
            if ((a[r] >> c) & 1u) {
                piv = r;
                break;
            }
        if (piv < 0) return false;
        std::swap(a[c], a[piv]);
        std::swap(e[c], e[piv]);
        for (int r = 0; r < n; ++r)
            if (r != c && ((a[r] >> c) & 1u)) {
                a[r] ^= a[c];
                e[r] ^= e[c];
            }
    }
    *inv = e;
    return true;
}

// y = M v over GF(2), M by rows
inline uint32_t gf2_apply(const std::vector<uint32_t> &rows, uint32_t v) {
    uint32_t y = 0;
    for (size_t j = 0; j < rows.size(); ++j) y |= uint32_t(popc(rows[j] & v) & 1) << j;
    return y;
}

// remove bit positions t1 < t2 from v
inline uint32_t drop2(uint32_t v, int t1, int t2) {
    const uint32_t lo1 = (1u << t1) - 1u;
    v = (v & lo1) | ((v >> 1) & ~lo1);  // bit t1 removed; t2 moved to t2 - 1
    const int u2 = t2 - 1;
    const uint32_t lo2 = (1u << u2) - 1u;
    return (v & lo2) | ((v >> 1) & ~lo2);
}

}  // namespace

namespace uccsd {

// Positions of the electron-sector determinants in the tapered encoding
// above, split by spin: the determinant with alpha orbital string sa and
// beta string sb sits at aoff[sa] + boff[sb] of the 2^(n-2) vector.  The
// tree's alpha nodes (below n/2 - 1) sum alpha orbitals only and its beta
// nodes (n/2 .. n - 2) beta orbitals only; the two nodes that mix or fix
// the parities are the tapered ones, so the kept alpha bits (positions
// 0 .. n/2 - 2) depend on sa alone and the kept beta bits (n/2 - 1 ..
// n - 3) on sb alone.
void scbk_addresses(int n_orb, std::vector<uint32_t> *aoff, std::vector<uint32_t> *boff) {
    const int n = 2 * n_orb, m = n_orb;
    const std::vector<uint32_t> B = bk_tree_rows(n);
    aoff->assign(size_t(1) << m, 0u);
    boff->assign(size_t(1) << m, 0u);
    for (uint32_t sv = 0; sv < (1u << m); ++sv) {
        (*aoff)[sv] = drop2(gf2_apply(B, sv), m - 1, n - 1);
        (*boff)[sv] = drop2(gf2_apply(B, sv << m), m - 1, n - 1);
    }
}

}  // namespace uccsd

extern "C" uccsd_status uccsd_pauli_terms_scbk(int n_orb, const double *h, const double *eri,
                                               double e_core, int n_alpha, int n_beta,
                                               uint32_t *xmask, uint32_t *zmask, double *coef,
                                               int cap, int *n_out, int *n_qubits_out) {
    if (n_orb < 2 || 2 * n_orb > 30 || !h || !eri || n_alpha < 0 || n_beta < 0 ||
        n_alpha > n_orb || n_beta > n_orb || cap < 0 || !n_out ||
        (cap > 0 && (!xmask || !zmask || !coef)))
        return UCCSD_ERR_ARG;
    for (size_t i = 0; i < size_t(n_orb) * n_orb; ++i)
        if (!std::isfinite(h[i])) return UCCSD_ERR_ARG;
    for (size_t i = 0; i < size_t(n_orb) * n_orb * n_orb * n_orb; ++i)
        if (!std::isfinite(eri[i])) return UCCSD_ERR_ARG;
    const int n = 2 * n_orb, m = n_orb;
    std::vector<int> qubit_of(n);
    for (int P = 0; P < n; ++P) qubit_of[P] = (P & 1) ? m + (P >> 1) : (P >> 1);
    std::vector<uccsd::XZTerm> terms;
    std::string err;
    if (!uccsd::pauli_terms_ordered(n_orb, h, eri, e_core, qubit_of.data(), &terms, &err))
        return UCCSD_ERR_ARG;
    const std::vector<uint32_t> B = bk_tree_rows(n);
    std::vector<uint32_t> Binv;
    if (!gf2_inverse(B, &Binv)) return UCCSD_ERR_ARG;
    // columns of B^-1 give B^-T z: (B^-T z)_j = parity(z & column j of B^-1)
    std::vector<uint32_t> BinvT(n, 0u);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if ((Binv[i] >> j) & 1u) BinvT[j] |= 1u << i;
    const int t1 = m - 1, t2 = n - 1;
    const double s1 = (n_alpha & 1) ? -1.0 : 1.0;              // Z on the alpha-parity qubit
    const double s2 = ((n_alpha + n_beta) & 1) ? -1.0 : 1.0;  // Z on the total-parity qubit
    std::map<uint64_t, double> acc;
    for (const uccsd::XZTerm &t : terms) {
        const uint32_t x = gf2_apply(B, t.x), z = gf2_apply(BinvT, t.z);
        if (((x >> t1) & 1u) || ((x >> t2) & 1u)) return UCCSD_ERR_ARG;  // not a symmetry
        double c = t.c;
        if ((z >> t1) & 1u) c *= s1;
        if ((z >> t2) & 1u) c *= s2;
        acc[(uint64_t(drop2(x, t1, t2)) << 32) | drop2(z, t1, t2)] += c;
    }
    double cmax = 0.0;
    for (const auto &kv : acc) cmax = std::max(cmax, std::fabs(kv.second));
    int count = 0;
    for (const auto &kv : acc) {
        if (!(std::fabs(kv.second) > 1e-13 * cmax)) continue;
        if (count < cap) {
            xmask[count] = uint32_t(kv.first >> 32);
            zmask[count] = uint32_t(kv.first);
            coef[count] = kv.second;
        }
        ++count;
    }
    *n_out = count;
    if (n_qubits_out) *n_qubits_out = n - 2;
    return UCCSD_OK;
}
