// Jordan-Wigner compiler (host).  Maps the second-quantised Hamiltonian of
// Eq. 2 and the UCCSD generators of Eq. 4 to real Pauli terms in the
// X^x Z^z form and groups the Hamiltonian terms by X-mask.
//
// Ladder operators (qubit P = spin orbital P, bit = occupation):
//   a_P   = Z^{<P} |0><1|_P = 1/2 X_P Z^{<P} - 1/2 X_P Z^{<P} Z_P
//   a+_P  = Z^{<P} |1><0|_P = 1/2 X_P Z^{<P} + 1/2 X_P Z^{<P} Z_P
// Product rule: (X^a Z^b)(X^c Z^d) = (-1)^{popc(b & c)} X^{a^c} Z^{b^d}.
// Every coefficient stays real, so the compiled H is a real matrix.
#include "jw.hpp"

#include <algorithm>
#include <cmath>
#include <unordered_map>

namespace uccsd {
namespace {

inline int popc(uint32_t v) { return __builtin_popcount(v); }

inline XZTerm mul(const XZTerm &a, const XZTerm &b) {
    double s = (popc(a.z & b.x) & 1) ? -1.0 : 1.0;
    return XZTerm{a.x ^ b.x, a.z ^ b.z, a.c * b.c * s};
}

inline void ladder(int p, bool dag, XZTerm out[2]) {
    uint32_t bp = 1u << p;
    uint32_t below = bp - 1u;
    out[0] = XZTerm{bp, below, 0.5};
    out[1] = XZTerm{bp, below | bp, dag ? 0.5 : -0.5};
}

// Expand coef * op[0] op[1] ... op[len-1] (matrix product, rightmost acts
// first) into X^x Z^z terms.
int expand(int len, const int *idx, const bool *dag, double coef, XZTerm *out) {
    int n = 1;
    out[0] = XZTerm{0u, 0u, coef};
    XZTerm tmp[16];
    for (int t = 0; t < len; ++t) {
        XZTerm l[2];
        ladder(idx[t], dag[t], l);
        int m = 0;
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 2; ++k) tmp[m++] = mul(out[i], l[k]);
        n = m;
        for (int i = 0; i < n; ++i) out[i] = tmp[i];
    }
    return n;
}

inline uint64_t key(uint32_t x, uint32_t z) { return (uint64_t(x) << 32) | z; }

// Open-addressing accumulator of X^x Z^z coefficients (linear probing,
// power-of-two capacity, splitmix64 finaliser as the hash).
class TermTable {
  public:
    explicit TermTable(size_t expected) {
        size_t cap = 64;
        while (cap < 2 * expected) cap <<= 1;
        keys_.assign(cap, kEmpty);
        vals_.assign(cap, 0.0);
        mask_ = cap - 1;
    }
    void add(uint64_t k, double v) {
        size_t i = hash(k) & mask_;
        while (keys_[i] != kEmpty && keys_[i] != k) i = (i + 1) & mask_;
        if (keys_[i] == kEmpty) {
            keys_[i] = k;
            if (++count_ * 2 > keys_.size()) {
                vals_[i] += v;
                grow();
                return;
            }
        }
        vals_[i] += v;
    }
    template <typename F>
    void each(F f) const {
        for (size_t i = 0; i < keys_.size(); ++i)
            if (keys_[i] != kEmpty) f(keys_[i], vals_[i]);
    }

  private:
    static constexpr uint64_t kEmpty = ~0ull;
    static uint64_t hash(uint64_t z) {
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    void grow() {
        std::vector<uint64_t> k2;
        std::vector<double> v2;
        k2.swap(keys_);
        v2.swap(vals_);
        keys_.assign(k2.size() * 2, kEmpty);
        vals_.assign(k2.size() * 2, 0.0);
        mask_ = keys_.size() - 1;
        for (size_t i = 0; i < k2.size(); ++i)
            if (k2[i] != kEmpty) {
                size_t j = hash(k2[i]) & mask_;
                while (keys_[j] != kEmpty) j = (j + 1) & mask_;
                keys_[j] = k2[i];
                vals_[j] = v2[i];
            }
    }
    std::vector<uint64_t> keys_;
    std::vector<double> vals_;
    size_t mask_ = 0, count_ = 0;
};

// Jordan-Wigner interval parity of a flip mask: bits outside the mask that
// lie below an odd number of the mask's bits.
uint32_t interval_mask(uint32_t x) {
    uint32_t m = 0;
    for (uint32_t v = x; v; v &= v - 1) m ^= (v & (~v + 1u)) - 1u;
    return m & ~x;
}

// Local pattern: bit k = bit pos[k] of y.
inline int pattern(uint32_t y, int nb, const int32_t *pos) {
    int p = 0;
    for (int k = 0; k < nb; ++k) p |= int((y >> pos[k]) & 1u) << k;
    return p;
}

}  // namespace

namespace {
// Eq. 2 as merged X^x Z^z terms, spin orbital P on qubit qubit_of[P]
// (Jordan-Wigner strings in qubit order), sorted by (x, z); merge residue
// |c| <= 1e-13 max|c| dropped.
std::vector<XZTerm> eq2_terms(int n_orb, const double *h, const double *eri, double e_core,
                              const int *qubit_of) {
    const int n = 2 * n_orb;
    // distinct keys: 16 Z-patterns per flip mask of 0, 2 or 4 bits
    const size_t n2 = size_t(n) * (n - 1) / 2, n4 = n2 * (n - 2) * (n - 3) / 12;
    TermTable acc(2 * (1 + n2 + n4));  // grows if needed
    XZTerm buf[16];
    auto add = [&](int cnt) {
        for (int i = 0; i < cnt; ++i) acc.add(key(buf[i].x, buf[i].z), buf[i].c);
    };
    // A + A^dagger of an expanded A: (X^x Z^z)^dagger = (-1)^{popc(x & z)} X^x Z^z,
    // so odd terms cancel and even terms double.
    auto add_hermitian = [&](int cnt) {
        for (int i = 0; i < cnt; ++i)
            if (!(popc(buf[i].x & buf[i].z) & 1)) acc.add(key(buf[i].x, buf[i].z), 2.0 * buf[i].c);
    };
    // one-body: sum_PQ h_PQ a+_P a_Q (same spin); h is symmetric, so the
    // pair P < Q is (a+_P a_Q) + its adjoint and P = Q stands alone
    for (int P = 0; P < n; ++P)
        for (int Q = P; Q < n; ++Q) {
            if ((P & 1) != (Q & 1)) continue;
            double c = h[(P >> 1) * n_orb + (Q >> 1)];
            if (c == 0.0) continue;
            int idx[2] = {qubit_of[P], qubit_of[Q]};
            bool dag[2] = {true, false};
            const int cnt = expand(2, idx, dag, c, buf);
            if (P == Q) add(cnt);
            else add_hermitian(cnt);
        }
    // two-body: 1/2 sum_PQRS <PQ|RS> a+_P a+_Q a_S a_R with <PQ|RS> = (pr|qs)
    // for spin(P) = spin(R), spin(Q) = spin(S), else 0.
    //  - (P,Q,R,S) and (Q,P,S,R) give the same operator and coefficient, so
    //    the sum runs over P < Q with weight 1 (P = Q vanishes);
    //  - a_R a_S = -a_S a_R, so (R,S) and (S,R) combine into R < S with
    //    coefficient c = <PQ|RS> - <PQ|SR>;
    //  - with real integrals the pair (R<S, P<Q) has the same c and the
    //    adjoint operator, so (P,Q) < (R,S) is expanded once as A + A^dagger
    //    and (P,Q) = (R,S) stands alone.
    auto g_of = [&](int P, int Q, int R, int S) {
        if ((P & 1) != (R & 1) || (Q & 1) != (S & 1)) return 0.0;
        const size_t p = P >> 1, q = Q >> 1, r = R >> 1, s = S >> 1;
        return eri[((p * n_orb + r) * n_orb + q) * n_orb + s];
    };
    for (int P = 0; P < n; ++P)
        for (int Q = P + 1; Q < n; ++Q)
            for (int R = P; R < n; ++R)
                for (int S = (R == P ? Q : R + 1); S < n; ++S) {
                    // spin conservation of the pair: N_alpha of (P,Q) = of (R,S)
                    if (((P & 1) + (Q & 1)) != ((R & 1) + (S & 1))) continue;
                    const double c = g_of(P, Q, R, S) - g_of(P, Q, S, R);
                    if (c == 0.0) continue;
                    int idx[4] = {qubit_of[P], qubit_of[Q], qubit_of[S], qubit_of[R]};
                    bool dag[4] = {true, true, false, false};
                    const int cnt = expand(4, idx, dag, c, buf);
                    if (R == P && S == Q) add(cnt);
                    else add_hermitian(cnt);
                }
    acc.add(key(0, 0), e_core);

    // merge residue: drop |c| <= 1e-13 max|c| (no approximate truncation)
    double cmax = 0.0;
    acc.each([&](uint64_t, double v) { cmax = std::max(cmax, std::fabs(v)); });
    std::vector<XZTerm> terms;
    acc.each([&](uint64_t k, double v) {
        if (std::fabs(v) > 1e-13 * cmax) terms.push_back(XZTerm{uint32_t(k >> 32), uint32_t(k), v});
    });
    std::sort(terms.begin(), terms.end(), [](const XZTerm &a, const XZTerm &b) {
        return a.x != b.x ? a.x < b.x : a.z < b.z;
    });
    return terms;
}
}  // namespace

bool pauli_terms_ordered(int n_orb, const double *h, const double *eri, double e_core,
                         const int *qubit_of, std::vector<XZTerm> *out, std::string *err) {
    if (n_orb < 1 || 2 * n_orb > 30) {
        *err = "n_orb out of range";
        return false;
    }
    *out = eq2_terms(n_orb, h, eri, e_core, qubit_of);
    return true;
}

bool compile_hamiltonian(int n_orb, const double *h, const double *eri, double e_core,
                         CompiledH *out, std::string *err) {
    const int n = 2 * n_orb;
    if (n_orb < 1 || n > 30) {
        *err = "n_orb out of range";
        return false;
    }
    std::vector<int> ident(n);
    for (int q = 0; q < n; ++q) ident[q] = q;
    std::vector<XZTerm> terms = eq2_terms(n_orb, h, eri, e_core, ident.data());

    CompiledH H;
    H.n_qubits = n;
    H.n_terms = int(terms.size());
    H.diag_a.assign(n, 0.0);
    H.diag_b.assign(size_t(n) * n, 0.0);
    uint32_t amask = 0;
    for (int q = 0; q < n; q += 2) amask |= 1u << q;

    size_t t = 0;
    while (t < terms.size()) {
        size_t e = t;
        while (e < terms.size() && terms[e].x == terms[t].x) ++e;
        uint32_t x = terms[t].x;
        if (x == 0) {
            // diagonal: (-1)^{popc(y&z)} with popc(z) <= 2 -> occupation form
            H.has_diag = true;
            for (size_t u = t; u < e; ++u) {
                uint32_t z = terms[u].z;
                double c = terms[u].c;
                int pz = popc(z);
                if (pz == 0) {
                    H.c0 += c;
                } else if (pz == 1) {
                    int q = __builtin_ctz(z);
                    H.c0 += c;
                    H.diag_a[q] -= 2.0 * c;
                } else if (pz == 2) {
                    int q = __builtin_ctz(z);
                    int r = 31 - __builtin_clz(z);
                    H.c0 += c;
                    H.diag_a[q] -= 2.0 * c;
                    H.diag_a[r] -= 2.0 * c;
                    H.diag_b[size_t(q) * n + r] += 4.0 * c;
                } else {
                    *err = "diagonal Pauli term with more than two Z";
                    return false;
                }
            }
        } else {
            GroupT<double> g{};
            g.xmask = x;
            g.nb = popc(x);
            if (g.nb != 2 && g.nb != 4) {
                *err = "X-mask group with an unexpected number of flipped bits";
                return false;
            }
            int k = 0;
            for (int q = 0; q < n; ++q)
                if ((x >> q) & 1u) g.pos[k++] = q;
            g.jmask = interval_mask(x);
            g.spec = -1;
            std::vector<double> spec;  // [w][pat]
            for (size_t u = t; u < e; ++u) {
                uint32_t z = terms[u].z;
                uint32_t d = (z & ~x) ^ g.jmask;
                int wl = pattern(z, g.nb, g.pos);
                double c = terms[u].c;
                if (d == 0) {
                    for (int p = 0; p < (1 << g.nb); ++p)
                        g.lut[p] += (popc(uint32_t(p & wl)) & 1) ? -c : c;
                } else if (popc(d) == 1 && g.nb == 2) {
                    if (spec.empty()) spec.assign(size_t(n) * 4, 0.0);
                    int w = __builtin_ctz(d);
                    for (int p = 0; p < 4; ++p)
                        spec[size_t(w) * 4 + p] += (popc(uint32_t(p & wl)) & 1) ? -c : c;
                } else {
                    *err = "Pauli term outside the interval/spectator structure";
                    return false;
                }
            }
            // (-1)^{y_w} = 1 - 2 y_w: fold the constant part into the LUT and
            // keep -2 * spec as the occupation-weighted spectator row.
            if (!spec.empty()) {
                for (int w = 0; w < n; ++w)
                    for (int p = 0; p < 4; ++p) {
                        g.lut[p] += spec[size_t(w) * 4 + p];
                        spec[size_t(w) * 4 + p] *= -2.0;
                    }
            }
            // Structural zeros: a pattern whose flip changes N_alpha or N_beta
            // has no matrix element.  Check the compiled value is round-off.
            double scale = 0.0;
            for (int p = 0; p < (1 << g.nb); ++p) scale = std::max(scale, std::fabs(g.lut[p]));
            for (int p = 0; p < (1 << g.nb); ++p) {
                int da = 0, db = 0;
                for (int b = 0; b < g.nb; ++b) {
                    int occ = (p >> b) & 1;
                    int dv = occ ? -1 : 1;  // flipping an occupied bit removes an electron
                    if ((amask >> g.pos[b]) & 1u) da += dv;
                    else db += dv;
                }
                if (da == 0 && db == 0) g.active |= 1u << p;
                if (da != 0 || db != 0) {
                    double r = std::fabs(g.lut[p]);
                    if (!spec.empty())
                        for (int w = 0; w < n; ++w) r += std::fabs(spec[size_t(w) * 4 + p]);
                    if (r > 1e-10 * std::max(1.0, scale)) {
                        *err = "compiled Hamiltonian does not conserve N_alpha/N_beta";
                        return false;
                    }
                    g.lut[p] = 0.0;
                    if (!spec.empty())
                        for (int w = 0; w < n; ++w) spec[size_t(w) * 4 + p] = 0.0;
                }
            }
            if (!spec.empty()) {
                g.spec = int(H.spec.size() / 4);
                H.spec.insert(H.spec.end(), spec.begin(), spec.end());
            }
            H.groups.push_back(g);
        }
        t = e;
    }
    H.terms = std::move(terms);
    *out = std::move(H);
    return true;
}

bool compile_excitation(int n_qubits, const int32_t *row, CompiledExc *out, std::string *err) {
    int i = row[0], j = row[1], a = row[2], b = row[3];
    bool single = j < 0;
    XZTerm buf[16], bufd[16];
    int cnt, cntd;
    if (single) {
        int idx[2] = {a, i};
        bool dag[2] = {true, false};
        cnt = expand(2, idx, dag, 1.0, buf);
        int idxd[2] = {i, a};
        cntd = expand(2, idxd, dag, -1.0, bufd);
    } else {
        int idx[4] = {a, b, j, i};
        bool dag[4] = {true, true, false, false};
        cnt = expand(4, idx, dag, 1.0, buf);
        int idxd[4] = {i, j, b, a};
        cntd = expand(4, idxd, dag, -1.0, bufd);
    }
    // merge G = tau - tau^dag
    std::unordered_map<uint64_t, double> acc;
    for (int t = 0; t < cnt; ++t) acc[key(buf[t].x, buf[t].z)] += buf[t].c;
    for (int t = 0; t < cntd; ++t) acc[key(bufd[t].x, bufd[t].z)] += bufd[t].c;
    uint32_t flip = 0, occ = 0;
    flip |= 1u << i;
    flip |= 1u << a;
    occ |= 1u << i;
    if (!single) {
        flip |= 1u << j;
        flip |= 1u << b;
        occ |= 1u << j;
    }
    int nb = popc(flip);
    if (nb != (single ? 2 : 4)) {
        *err = "excitation indices are not distinct";
        return false;
    }
    int32_t pos[4] = {0, 0, 0, 0};
    int k = 0;
    for (int q = 0; q < n_qubits; ++q)
        if ((flip >> q) & 1u) pos[k++] = q;
    uint32_t J = interval_mask(flip);
    double lut[16] = {0};
    for (auto &kv : acc) {
        uint32_t x = uint32_t(kv.first >> 32), z = uint32_t(kv.first);
        if (kv.second == 0.0) continue;
        if (x != flip || ((z & ~flip) != J)) {
            *err = "generator term outside the interval structure";
            return false;
        }
        int wl = pattern(z, nb, pos);
        for (int p = 0; p < (1 << nb); ++p) lut[p] += (popc(uint32_t(p & wl)) & 1) ? -kv.second : kv.second;
    }
    int po = pattern(occ, nb, pos);
    int pe = pattern(flip & ~occ, nb, pos);
    double s_occ = lut[po], s_emp = lut[pe];
    if (std::fabs(std::fabs(s_occ) - 1.0) > 1e-12 || std::fabs(s_emp + s_occ) > 1e-12) {
        *err = "generator sign table is not antisymmetric +-1";
        return false;
    }
    for (int p = 0; p < (1 << nb); ++p)
        if (p != po && p != pe && std::fabs(lut[p]) > 1e-12) {
            *err = "generator acts outside its pair";
            return false;
        }
    out->flip = flip;
    out->occ = occ;
    out->par = J;
    out->s0 = s_occ > 0 ? 1 : -1;
    out->nb = nb;
    return true;
}

}  // namespace uccsd
