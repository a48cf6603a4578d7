#include "plan.hpp"

#include <algorithm>

namespace uccsd {
namespace {
inline int popc(uint32_t v) { return __builtin_popcount(v); }

// Gather the bits of v selected by mask into the low bits (software pext).
uint32_t gather_bits(uint32_t v, uint32_t mask) {
    uint32_t r = 0;
    int k = 0;
    for (uint32_t m = mask; m; m &= m - 1) {
        int b = __builtin_ctz(m);
        r |= ((v >> b) & 1u) << k++;
    }
    return r;
}
}  // namespace

uint64_t hf_bits(int n_alpha, int n_beta) {
    uint64_t x = 0;
    for (int p = 0; p < n_alpha; ++p) x |= 1ull << (2 * p);
    for (int p = 0; p < n_beta; ++p) x |= 1ull << (2 * p + 1);
    return x;
}

std::vector<int32_t> build_uccsd_list(int n_orb, int n_alpha, int n_beta) {
    const int n = 2 * n_orb;
    uint64_t hf = hf_bits(n_alpha, n_beta);
    std::vector<int> occ, vir;
    for (int q = 0; q < n; ++q) ((hf >> q) & 1u ? occ : vir).push_back(q);
    std::vector<int32_t> out;
    for (int i : occ)
        for (int a : vir)
            if ((i & 1) == (a & 1)) out.insert(out.end(), {i, -1, a, -1});
    for (size_t ii = 0; ii < occ.size(); ++ii)
        for (size_t jj = ii + 1; jj < occ.size(); ++jj)
            for (size_t aa = 0; aa < vir.size(); ++aa)
                for (size_t bb = aa + 1; bb < vir.size(); ++bb) {
                    int i = occ[ii], j = occ[jj], a = vir[aa], b = vir[bb];
                    // spin multiset {s_i, s_j} == {s_a, s_b}
                    if ((i & 1) + (j & 1) == (a & 1) + (b & 1))
                        out.insert(out.end(), {i, j, a, b});
                }
    return out;
}

void build_schedule(int K, int order, int M, std::vector<int32_t> *op_k,
                    std::vector<double> *op_scale) {
    op_k->clear();
    op_scale->clear();
    for (int m = 0; m < M; ++m) {
        if (order == 1) {
            for (int k = 0; k < K; ++k) {
                op_k->push_back(k);
                op_scale->push_back(1.0 / M);
            }
        } else {
            for (int k = 0; k < K; ++k) {
                op_k->push_back(k);
                op_scale->push_back(0.5 / M);
            }
            for (int k = K - 1; k >= 0; --k) {
                op_k->push_back(k);
                op_scale->push_back(0.5 / M);
            }
        }
    }
}

namespace {
long long binom(int m, int k) {
    if (k < 0 || k > m) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (m - k + i) / i;
    return r;
}

// Largest C(L, a) over the electron counts a that a tile with L bits of one
// spin can hold when the other N_spin - L bits of that spin carry the rest.
long long max_binom(int L, int n_spin_bits, int n_el) {
    int lo = std::max(0, n_el - (n_spin_bits - L)), hi = std::min(L, n_el);
    long long m = 0;
    for (int a = lo; a <= hi; ++a) m = std::max(m, binom(L, a));
    return m;
}

uint32_t deposit_bits(uint32_t v, uint32_t mask) {
    uint32_t r = 0;
    for (uint32_t m = mask; m; m &= m - 1) {
        if (v & 1u) r |= m & (~m + 1u);
        v >>= 1;
    }
    return r;
}
}  // namespace

void max_tile_sides(int n_qubits, int n_alpha, int n_beta, uint32_t tmask, long long *da,
                    long long *db) {
    uint32_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1u << q;
    const uint32_t bmask = ((n_qubits >= 32) ? 0xFFFFFFFFu : ((1u << n_qubits) - 1u)) & ~amask;
    *da = max_binom(popc(tmask & amask), popc(amask), n_alpha);
    *db = max_binom(popc(tmask & bmask), popc(bmask), n_beta);
}

size_t sweep_smem_bytes(long long entries, long long da, long long db, size_t amp_bytes,
                        int nvec, int n_ops_run, int lmax) {
    size_t b = size_t(tile_alloc(entries)) * amp_bytes * nvec + 2 * size_t(da + db) * 8 +
               size_t(n_ops_run) * (sizeof(COpDev) + amp_bytes + 8);
    if (lmax <= kStageLmax) b += sweep_table_bytes(lmax);
    return b;
}

size_t sweep_table_bytes(int lmax) {
    // combos and ranks prefixes (bit counts <= lmax) and their class offsets
    return 2 * (((size_t(1) << (lmax + 1)) - 1) * sizeof(uint16_t)) +
           size_t(lmax + 1) * 17 * sizeof(int32_t) + 16;
}

long long max_tile_entries(int n_qubits, int n_alpha, int n_beta, uint32_t tmask) {
    uint32_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1u << q;
    const uint32_t bmask = ((n_qubits >= 32) ? 0xFFFFFFFFu : ((1u << n_qubits) - 1u)) & ~amask;
    const int La = popc(tmask & amask), Lb = popc(tmask & bmask);
    const int Na = popc(amask), Nb = popc(bmask);
    return max_binom(La, Na, n_alpha) * max_binom(Lb, Nb, n_beta);
}

SweepPlan plan_sweep(int n_qubits, int n_alpha, int n_beta, size_t amp_bytes, int nvec,
                     size_t budget, const std::vector<CompiledExc> &exc,
                     const std::vector<int32_t> &op_k) {
    SweepPlan plan;
    uint32_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1u << q;
    const uint32_t all = (n_qubits >= 32) ? 0xFFFFFFFFu : ((1u << n_qubits) - 1u);
    const uint32_t bmask = all & ~amask;
    auto fits = [&](uint32_t T, int run_ops) {
        long long da, db;
        max_tile_sides(n_qubits, n_alpha, n_beta, T, &da, &db);
        const int lmax = std::max(popc(T & amask), popc(T & bmask));
        return sweep_smem_bytes(max_tile_entries(n_qubits, n_alpha, n_beta, T), da, db,
                                amp_bytes, nvec, run_ops, lmax) <= budget;
    };
    plan.op_tiles.assign(op_k.size(), 1);
    size_t o = 0;
    const size_t n_ops = op_k.size();
    while (o < n_ops) {
        uint32_t U = exc[op_k[o]].flip;
        size_t e = o + 1;
        while (e < n_ops && fits(U | exc[op_k[e]].flip, int(e - o + 1))) {
            U |= exc[op_k[e]].flip;
            ++e;
        }
        CRunDev r{};
        r.emap_base = -1;
        r.pl_base = -1;
        r.tmask = U;
        r.rmask = all & ~U;
        const uint32_t Ta = U & amask, Tb = U & bmask;
        r.La = popc(Ta);
        r.Lb = popc(Tb);
        r.n_tiles = 1 << (n_qubits - r.La - r.Lb);
        r.max_entries = int(max_tile_entries(n_qubits, n_alpha, n_beta, U));
        {
            long long da, db;
            max_tile_sides(n_qubits, n_alpha, n_beta, U, &da, &db);
            r.max_da = int(da);
            r.max_db = int(db);
        }
        r.spread_off = int(plan.spread.size());
        // tile string -> orbital string (alpha: orbital t for qubit 2t; beta: qubit 2t + 1)
        for (uint32_t sidx = 0; sidx < (1u << r.La); ++sidx)
            plan.spread.push_back(gather_bits(deposit_bits(sidx, Ta), amask));
        for (uint32_t sidx = 0; sidx < (1u << r.Lb); ++sidx)
            plan.spread.push_back(gather_bits(deposit_bits(sidx, Tb), bmask));
        r.op_begin = int(plan.ops.size());
        for (size_t u = o; u < e; ++u) {
            const CompiledExc &x = exc[op_k[u]];
            COpDev d{};
            d.fa = gather_bits(x.flip, Ta);
            d.fb = gather_bits(x.flip, Tb);
            d.oa = gather_bits(x.occ, Ta);
            d.ob = gather_bits(x.occ, Tb);
            d.pa = gather_bits(x.par, Ta);
            d.pb = gather_bits(x.par, Tb);
            d.par_rest = x.par & ~U;
            d.op_s0 = uint32_t(u) | (x.s0 < 0 ? 0x80000000u : 0u);
            plan.ops.push_back(d);
            plan.op_tiles[u] = r.n_tiles;
        }
        r.op_end = int(plan.ops.size());
        plan.max_tiles = std::max(plan.max_tiles, r.n_tiles);
        plan.max_entries = std::max(plan.max_entries, r.max_entries);
        plan.runs.push_back(r);
        o = e;
    }
    return plan;
}

namespace {
// Insert a zero bit at each set bit position of mask, lowest first.
uint32_t insert_zeros_host(uint32_t j, uint32_t mask) {
    for (; mask; mask &= mask - 1u) {
        const uint32_t lowm = (mask & (0u - mask)) - 1u;
        j = ((j & ~lowm) << 1) | (j & lowm);
    }
    return j;
}
}  // namespace

namespace {
// Conflict-free grouping of one factor's pairs.  With G lanes served by one
// shared-memory wavefront, pair (e, e') is an edge between residue e mod G
// (left) and e' mod G (right) of a bipartite multigraph; a proper edge
// colouring puts at most one pair of each left and each right residue in a
// colour, so every colour class is a conflict-free group.  A bipartite
// multigraph of maximum degree D has a proper D-colouring (Konig); it is
// built edge by edge, swapping two colours along an alternating path when
// the endpoints have no common free colour.  Each class is padded to G
// pairs with dummy pairs on zeroed scratch entries scratch + r (e side) and
// scratch + G + r (e' side) for residues r unused by the class.  Returns the
// padded list (2 words per pair).
std::vector<uint32_t> bank_groups(const uint32_t *pairs, int P, int G, uint32_t scratch) {
    std::vector<uint32_t> out;
    if (P <= 0) return out;
    std::vector<int> deg(2 * G, 0);
    for (int i = 0; i < P; ++i) {
        deg[(pairs[2 * i] & 0x7FFFFFFFu) % G]++;
        deg[G + pairs[2 * i + 1] % G]++;
    }
    const int D = *std::max_element(deg.begin(), deg.end());
    // at[node * D + c] = edge of colour c at node, or -1
    std::vector<int> at(size_t(2 * G) * D, -1), col(P, -1), eu(P), ev(P);
    for (int i = 0; i < P; ++i) {
        eu[i] = int((pairs[2 * i] & 0x7FFFFFFFu) % G);
        ev[i] = G + int(pairs[2 * i + 1] % G);
    }
    auto free_col = [&](int node) {
        for (int c = 0; c < D; ++c)
            if (at[size_t(node) * D + c] < 0) return c;
        return -1;
    };
    for (int i = 0; i < P; ++i) {
        const int u = eu[i], v = ev[i];
        const int a = free_col(u), b = free_col(v);
        if (at[size_t(v) * D + a] >= 0) {
            // a is used at v: swap a and b along the path from v that starts
            // with its a-edge (it cannot reach u, so a becomes free at v)
            std::vector<int> path;
            int node = v, c = a;
            for (;;) {
                const int ed = at[size_t(node) * D + c];
                if (ed < 0) break;
                path.push_back(ed);
                node = (node == eu[ed]) ? ev[ed] : eu[ed];
                c = (c == a) ? b : a;
            }
            for (int ed : path) {
                at[size_t(eu[ed]) * D + col[ed]] = -1;
                at[size_t(ev[ed]) * D + col[ed]] = -1;
            }
            for (int ed : path) {
                col[ed] = (col[ed] == a) ? b : a;
                at[size_t(eu[ed]) * D + col[ed]] = ed;
                at[size_t(ev[ed]) * D + col[ed]] = ed;
            }
        }
        col[i] = a;
        at[size_t(u) * D + a] = i;
        at[size_t(v) * D + a] = i;
    }
    out.reserve(size_t(2) * D * G);
    for (int c = 0; c < D; ++c) {
        uint32_t used_e = 0, used_f = 0;
        int m = 0;
        for (int r = 0; r < G; ++r) {
            const int ed = at[size_t(r) * D + c];
            if (ed < 0) continue;
            out.push_back(pairs[2 * ed]);
            out.push_back(pairs[2 * ed + 1]);
            used_e |= 1u << eu[ed];
            used_f |= 1u << (ev[ed] - G);
            ++m;
        }
        for (int re = 0, rf = 0; m < G; ++m) {
            while (used_e >> re & 1u) ++re;
            while (used_f >> rf & 1u) ++rf;
            out.push_back(scratch + uint32_t(re++));
            out.push_back(scratch + uint32_t(G + rf++));
        }
    }
    return out;
}
}  // namespace

bool build_pair_lists(int n_qubits, int n_alpha, int n_beta, size_t max_pairs, SweepPlan *plan,
                      PairLists *out, int bank_group) {
    std::vector<uint16_t> combos, rank;
    std::vector<int32_t> offs;
    build_comb_tables(&combos, &rank, &offs);
    auto cnt = [&](int m, int k) { return (k < 0 || k > m) ? 0 : offs[m * 17 + k + 1] - offs[m * 17 + k]; };
    auto strings = [&](int m, int k) { return &combos[((size_t(1) << m) - 1) + offs[m * 17 + k]]; };
    uint32_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1u << q;
    // size first
    size_t total = 0, n_pl = 0;
    for (const CRunDev &r : plan->runs) {
        const int nops = r.op_end - r.op_begin;
        const int ra = popc(r.rmask & amask), rb = popc(r.rmask & ~amask);
        n_pl += size_t(r.La + 1) * (r.Lb + 1) * nops;
        for (int a = 0; a <= r.La; ++a)
            for (int b = 0; b <= r.Lb; ++b) {
                if (n_alpha - a < 0 || n_alpha - a > ra || n_beta - b < 0 || n_beta - b > rb) continue;
                for (int o = r.op_begin; o < r.op_end; ++o) {
                    const COpDev &op = plan->ops[o];
                    total += size_t(cnt(r.La - popc(op.fa), a - popc(op.oa))) *
                             size_t(cnt(r.Lb - popc(op.fb), b - popc(op.ob)));
                }
            }
    }
    if (total > max_pairs) {
        for (CRunDev &r : plan->runs) r.pl_base = -1;
        return false;
    }
    out->pairs.clear();
    out->pairs.reserve(2 * total + 2 * total / 4);
    out->op_pl.assign(2 * n_pl, 0);
    size_t pos = 0, plb = 0;
    std::vector<uint32_t> raw;
    std::vector<uint32_t> ea, ea2, eb, eb2;
    std::vector<uint8_t> pa_, pb_;
    for (CRunDev &r : plan->runs) {
        const int nops = r.op_end - r.op_begin;
        const int ra = popc(r.rmask & amask), rb = popc(r.rmask & ~amask);
        r.pl_base = int32_t(plb);
        const uint16_t *rka = &rank[(size_t(1) << r.La) - 1];
        const uint16_t *rkb = &rank[(size_t(1) << r.Lb) - 1];
        for (int a = 0; a <= r.La; ++a)
            for (int b = 0; b <= r.Lb; ++b) {
                const size_t cbase = plb + (size_t(a) * (r.Lb + 1) + b) * nops;
                if (n_alpha - a < 0 || n_alpha - a > ra || n_beta - b < 0 || n_beta - b > rb) continue;
                const uint32_t Db = uint32_t(cnt(r.Lb, b));
                for (int o = 0; o < nops; ++o) {
                    const COpDev &op = plan->ops[r.op_begin + o];
                    const int ma = r.La - popc(op.fa), ka = a - popc(op.oa);
                    const int mb = r.Lb - popc(op.fb), kb = b - popc(op.ob);
                    const int Va = cnt(ma, ka), Vb = cnt(mb, kb);
                    out->op_pl[2 * (cbase + o)] = int32_t(pos);
                    out->op_pl[2 * (cbase + o) + 1] = 0;
                    if (!Va || !Vb) continue;
                    ea.resize(Va); ea2.resize(Va); pa_.resize(Va);
                    eb.resize(Vb); eb2.resize(Vb); pb_.resize(Vb);
                    const uint16_t *fa = strings(ma, ka), *fb = strings(mb, kb);
                    for (int i = 0; i < Va; ++i) {
                        const uint32_t sv = insert_zeros_host(fa[i], op.fa) | op.oa;
                        ea[i] = uint32_t(rka[sv]) * Db;
                        ea2[i] = uint32_t(rka[sv ^ op.fa]) * Db;
                        pa_[i] = uint8_t(popc(sv & op.pa) & 1);
                    }
                    for (int i = 0; i < Vb; ++i) {
                        const uint32_t sv = insert_zeros_host(fb[i], op.fb) | op.ob;
                        eb[i] = rkb[sv];
                        eb2[i] = rkb[sv ^ op.fb];
                        pb_[i] = uint8_t(popc(sv & op.pb) & 1);
                    }
                    // A pair with odd string parity rotates as the pair with
                    // its entries swapped and even parity: store it that way,
                    // so the kernels apply no per-pair sign.
                    raw.resize(2 * size_t(Va) * Vb);
                    size_t q = 0;
                    for (int i = 0; i < Va; ++i)
                        for (int j = 0; j < Vb; ++j) {
                            const uint32_t e = ea[i] + eb[j], e2 = ea2[i] + eb2[j];
                            const bool odd = (pa_[i] ^ pb_[j]) & 1;
                            raw[q++] = odd ? e2 : e;
                            raw[q++] = odd ? e : e2;
                        }
                    const std::vector<uint32_t> g =
                        bank_groups(raw.data(), Va * Vb, bank_group, tile_scratch(r.max_entries));
                    out->pairs.insert(out->pairs.end(), g.begin(), g.end());
                    out->op_pl[2 * (cbase + o) + 1] = int32_t(g.size() / 2);
                    pos += g.size() / 2;
                }
            }
        plb += size_t(r.La + 1) * (r.Lb + 1) * nops;
    }
    out->n_pairs = pos;
    return true;
}

std::vector<ExpandedPair> expand_pair_lists(int n_qubits, int n_alpha, int n_beta,
                                            const SweepPlan &plan, const PairLists &L) {
    std::vector<uint16_t> combos, rank;
    std::vector<int32_t> offs;
    build_comb_tables(&combos, &rank, &offs);
    auto cnt = [&](int m, int k) { return (k < 0 || k > m) ? 0 : offs[m * 17 + k + 1] - offs[m * 17 + k]; };
    auto strings = [&](int m, int k) { return &combos[((size_t(1) << m) - 1) + offs[m * 17 + k]]; };
    uint32_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1u << q;
    std::vector<ExpandedPair> out;
    for (const CRunDev &r : plan.runs) {
        if (r.pl_base < 0) continue;
        const int nops = r.op_end - r.op_begin;
        const uint32_t Ta = r.tmask & amask, Tb = r.tmask & ~amask;
        const uint32_t scratch = uint32_t(tile_scratch(r.max_entries));
        for (int t = 0; t < r.n_tiles; ++t) {
            const uint32_t rest = deposit_bits(uint32_t(t), r.rmask);
            const int a = n_alpha - popc(rest & amask), b = n_beta - popc(rest & ~amask);
            if (a < 0 || a > r.La || b < 0 || b > r.Lb) continue;
            const int cls = a * (r.Lb + 1) + b;
            const uint32_t Db = uint32_t(cnt(r.Lb, b));
            const uint16_t *sa = strings(r.La, a), *sb = strings(r.Lb, b);
            auto det = [&](uint32_t e) {
                return rest | deposit_bits(sa[e / Db], Ta) | deposit_bits(sb[e % Db], Tb);
            };
            for (int o = 0; o < nops; ++o) {
                const COpDev &op = plan.ops[r.op_begin + o];
                const size_t slot = size_t(r.pl_base) + size_t(cls) * nops + o;
                const int32_t pos = L.op_pl[2 * slot], n = L.op_pl[2 * slot + 1];
                int sign = (op.op_s0 & 0x80000000u) ? -1 : 1;
                if (popc(rest & op.par_rest) & 1) sign = -sign;
                for (int j = 0; j < n; ++j) {
                    const uint32_t w0 = L.pairs[2 * (size_t(pos) + j)], w1 = L.pairs[2 * (size_t(pos) + j) + 1];
                    ExpandedPair x;
                    x.factor = int32_t(op.op_s0 & 0x7FFFFFFFu);
                    x.sign = sign;
                    x.e = int32_t(w0);
                    x.e2 = int32_t(w1);
                    x.index = j;
                    const bool pad = w0 >= scratch || w1 >= scratch;
                    x.first = pad ? 0xFFFFFFFFu : det(w0);
                    x.second = pad ? 0xFFFFFFFFu : det(w1);
                    out.push_back(x);
                }
            }
        }
    }
    return out;
}

std::vector<uint32_t> build_entry_map(int n_qubits, int n_alpha, int n_beta, SweepPlan *plan) {
    size_t total = 0;
    for (CRunDev &r : plan->runs) total += size_t(r.n_tiles) * size_t(r.max_entries);
    const int no = n_qubits / 2;
    std::vector<uint32_t> rank(size_t(1) << no);
    std::vector<int> cnt(no + 2, 0);
    for (uint32_t sv = 0; sv < (1u << no); ++sv) rank[sv] = uint32_t(cnt[popc(sv)]++);
    const uint32_t dbs = uint32_t(cnt[n_beta]);  // C(n_orb, n_beta)
    uint32_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1u << q;
    auto strings = [](int L, int k) {  // L-bit strings of popcount k, ascending
        std::vector<uint32_t> v;
        for (uint32_t s = 0; s < (1u << L); ++s)
            if (popc(s) == k) v.push_back(s);
        return v;
    };
    std::vector<uint32_t> map(total, 0u);
    size_t base = 0;
    for (CRunDev &r : plan->runs) {
        r.emap_base = int32_t(base);
        const uint32_t *spa = plan->spread.data() + r.spread_off;
        const uint32_t *spb = spa + (size_t(1) << r.La);
        for (int bx = 0; bx < r.n_tiles; ++bx) {
            const uint32_t rest = deposit_bits(uint32_t(bx), r.rmask);
            const int a = n_alpha - popc(rest & amask), b = n_beta - popc(rest & ~amask);
            if (a < 0 || a > r.La || b < 0 || b > r.Lb) continue;
            uint32_t ra = 0, rb = 0;  // orbital strings of the rest bits
            for (uint32_t m = rest; m; m &= m - 1u) {
                const int q = __builtin_ctz(m);
                if (q & 1) rb |= 1u << (q >> 1);
                else ra |= 1u << (q >> 1);
            }
            const std::vector<uint32_t> sa = strings(r.La, a), sb = strings(r.Lb, b);
            uint32_t *m = map.data() + base + size_t(bx) * size_t(r.max_entries);
            for (size_t ia = 0; ia < sa.size(); ++ia) {
                const uint32_t xa = rank[ra | spa[sa[ia]]] * dbs;
                for (size_t ib = 0; ib < sb.size(); ++ib) m[ia * sb.size() + ib] = xa + rank[rb | spb[sb[ib]]];
            }
        }
        base += size_t(r.n_tiles) * size_t(r.max_entries);
    }
    return map;
}

std::vector<uint32_t> tile_entry_dets(int n_qubits, int n_alpha, int n_beta, const CRunDev &r,
                                      int tile) {
    uint32_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1u << q;
    const uint32_t rest = deposit_bits(uint32_t(tile), r.rmask);
    const int a = n_alpha - popc(rest & amask), b = n_beta - popc(rest & ~amask);
    std::vector<uint32_t> out;
    if (a < 0 || a > r.La || b < 0 || b > r.Lb) return out;
    const uint32_t Ta = r.tmask & amask, Tb = r.tmask & ~amask;
    for (uint32_t s = 0; s < (1u << r.La); ++s) {
        if (popc(s) != a) continue;
        for (uint32_t t = 0; t < (1u << r.Lb); ++t)
            if (popc(t) == b) out.push_back(rest | deposit_bits(s, Ta) | deposit_bits(t, Tb));
    }
    return out;
}

void build_comb_tables(std::vector<uint16_t> *combos, std::vector<uint16_t> *rank,
                       std::vector<int32_t> *offs) {
    combos->assign((size_t(1) << (kCombMax + 1)) - 1, 0);
    rank->assign(combos->size(), 0);
    offs->assign(size_t(kCombMax + 1) * 17, 0);
    for (int m = 0; m <= kCombMax; ++m) {
        const size_t base = (size_t(1) << m) - 1;
        size_t pos = 0;
        for (int c = 0; c <= m; ++c) {
            (*offs)[m * 17 + c] = int32_t(pos);
            int32_t r = 0;
            for (uint32_t s = 0; s < (1u << m); ++s)
                if (popc(s) == c) {
                    (*combos)[base + pos++] = uint16_t(s);
                    (*rank)[base + s] = uint16_t(r++);
                }
        }
        (*offs)[m * 17 + m + 1] = int32_t(pos);
    }
}

namespace {
// Minimum-cost perfect matching of rows to columns of an n x n cost matrix
// (row-major) by successive shortest augmenting paths: Dijkstra over the
// alternating paths on reduced costs C - u(row) - v(column), which the
// potential update keeps non-negative, and zero on matched edges.  Returns
// the column of each row.
std::vector<int> min_cost_assignment(int n, const std::vector<int> &C) {
    const long long kInf = 1LL << 60;
    std::vector<long long> u(n), v(n, 0), dist(n), drow(n);
    std::vector<int> row_to(n, -1), col_to(n, -1), via(n);
    std::vector<char> done(n);
    for (int i = 0; i < n; ++i) u[i] = *std::min_element(C.begin() + size_t(i) * n, C.begin() + size_t(i + 1) * n);
    for (int s = 0; s < n; ++s) {
        std::fill(done.begin(), done.end(), 0);
        std::fill(drow.begin(), drow.end(), kInf);
        drow[s] = 0;
        for (int j = 0; j < n; ++j) {
            dist[j] = C[size_t(s) * n + j] - u[s] - v[j];
            via[j] = s;
        }
        int jf = -1;
        for (;;) {
            int j = -1;
            for (int k = 0; k < n; ++k)
                if (!done[k] && (j < 0 || dist[k] < dist[j])) j = k;
            done[j] = 1;
            if (col_to[j] < 0) {
                jf = j;
                break;
            }
            const int i = col_to[j];  // through its matched row (reduced cost 0)
            drow[i] = dist[j];
            for (int k = 0; k < n; ++k) {
                if (done[k]) continue;
                const long long d = dist[j] + C[size_t(i) * n + k] - u[i] - v[k];
                if (d < dist[k]) {
                    dist[k] = d;
                    via[k] = i;
                }
            }
        }
        const long long D = dist[jf];
        for (int i = 0; i < n; ++i)
            if (drow[i] < kInf) u[i] += D - drow[i];
        for (int j = 0; j < n; ++j)
            if (done[j]) v[j] -= D - dist[j];
        // flip the path: column jf to the row it was reached from, that row's
        // old column to the row before it, back to row s
        for (int j = jf;;) {
            const int i = via[j];
            const int old = row_to[i];
            row_to[i] = j;
            col_to[j] = i;
            if (i == s) break;
            j = old;
        }
    }
    return row_to;
}

// Shared-memory wavefronts of one slot of the mixed loop for the lanes of
// an aligned group of eight columns: its 16-byte loads of the table item and
// of the source chunk each take as many wavefronts as the largest number of
// distinct items (sources) in one of the eight 16-byte bank groups.
int slot_wavefronts(const uint32_t *item, const uint32_t *src, int m) {
    int cnt_i[8] = {0}, cnt_s[8] = {0}, wi = 0, ws = 0;
    for (int a = 0; a < m; ++a) {
        bool seen_i = false, seen_s = false;
        for (int b = 0; b < a; ++b) {
            seen_i |= item[b] == item[a];
            seen_s |= src[b] == src[a];
        }
        if (!seen_i) wi = std::max(wi, ++cnt_i[item[a] & 7u]);
        if (!seen_s) ws = std::max(ws, ++cnt_s[src[a] & 7u]);
    }
    return wi + 2 * ws;  // the source item is two 16-byte chunks
}
}  // namespace

#ifndef UCCSD_MIXED_ORDER_ROUNDS
#define UCCSD_MIXED_ORDER_ROUNDS 8
#endif
constexpr int kMixedOrderRounds = UCCSD_MIXED_ORDER_ROUNDS;

std::vector<uint8_t> happly_mixed_order(int n_orb, int n_beta) {
    std::vector<uint32_t> bstr, rank(size_t(1) << n_orb, 0u);
    for (uint32_t s = 0; s < (1u << n_orb); ++s)
        if (popc(s) == n_beta) {
            rank[s] = uint32_t(bstr.size());
            bstr.push_back(s);
        }
    const int Db = int(bstr.size());
    const int ns = n_beta * (n_orb - n_beta);
    std::vector<uint8_t> order(size_t(ns) * Db);
    for (int t = 0; t < ns; ++t)
        for (int c = 0; c < Db; ++c) order[size_t(t) * Db + c] = uint8_t(t);
    if (ns < 2) return order;
    // natural entries of each column: table item and source rank of its
    // k-th single j -> b (j occupied ascending, then b empty ascending)
    std::vector<uint32_t> item(size_t(Db) * ns), src(size_t(Db) * ns);
    for (int c = 0; c < Db; ++c) {
        const uint32_t sb = bstr[c];
        int k = 0;
        for (int j = 0; j < n_orb; ++j) {
            if (!((sb >> j) & 1u)) continue;
            for (int b = 0; b < n_orb; ++b) {
                if ((sb >> b) & 1u) continue;
                const int lo = std::min(j, b), hi = std::max(j, b);
                const uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
                const uint32_t pi = uint32_t(popc(sb & between) & 1);
                item[size_t(c) * ns + k] = uint32_t(j * n_orb + b) + uint32_t(n_orb * n_orb) * pi;
                src[size_t(c) * ns + k] = rank[sb ^ (1u << j) ^ (1u << b)];
                ++k;
            }
        }
    }
    std::vector<int> cost(size_t(ns) * ns);
    uint32_t ti[8], ts[8];
    for (int q0 = 0; q0 < Db; q0 += 8) {
        const int m = std::min(8, Db - q0);
        // coordinate descent: each column's singles re-assigned to the slots
        // by an exact minimum-cost assignment against the other columns of
        // the group (never worse than its current order; an equal-cost
        // assignment is taken too, which lets later columns move), a fixed
        // number of rounds
        for (int round = 0; round < kMixedOrderRounds; ++round) {
            for (int a = 0; a < m; ++a) {
                const int c = q0 + a;
                for (int t = 0; t < ns; ++t) {
                    for (int b = 0; b < m; ++b) {
                        const int k = order[size_t(t) * Db + q0 + b];
                        ti[b] = item[size_t(q0 + b) * ns + k];
                        ts[b] = src[size_t(q0 + b) * ns + k];
                    }
                    for (int k = 0; k < ns; ++k) {
                        ti[a] = item[size_t(c) * ns + k];
                        ts[a] = src[size_t(c) * ns + k];
                        cost[size_t(k) * ns + t] = slot_wavefronts(ti, ts, m);
                    }
                }
                const std::vector<int> slot = min_cost_assignment(ns, cost);
                for (int k = 0; k < ns; ++k) order[size_t(slot[k]) * Db + c] = uint8_t(k);
            }
        }
    }
    return order;
}

}  // namespace uccsd
