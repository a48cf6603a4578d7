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
    size_t b = size_t(entries) * amp_bytes * nvec + 2 * size_t(da + db) * 8 +
               size_t(n_ops_run) * (sizeof(COpDev) + amp_bytes);
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

}  // namespace uccsd
