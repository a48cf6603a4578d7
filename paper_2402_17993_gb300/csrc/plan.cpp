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

SweepPlan plan_sweep(int n_qubits, int L, int c_min, const std::vector<CompiledExc> &exc,
                     const std::vector<int32_t> &op_k) {
    SweepPlan plan;
    L = std::min(L, n_qubits);
    c_min = std::min(c_min, L);
    plan.L = L;
    const uint32_t all = (n_qubits >= 32) ? 0xFFFFFFFFu : ((1u << n_qubits) - 1u);
    const uint32_t low = (1u << c_min) - 1u;
    size_t o = 0;
    const size_t n_ops = op_k.size();
    while (o < n_ops) {
        uint32_t U = low;
        size_t e = o;
        while (e < n_ops) {
            uint32_t V = U | exc[op_k[e]].flip;
            if (popc(V) > L) break;
            U = V;
            ++e;
        }
        // pad with the lowest unused bits
        for (int q = 0; q < n_qubits && popc(U) < L; ++q) U |= 1u << q;
        RunDev r{};
        r.tmask = U;
        r.rmask = all & ~U;
        r.L = popc(U);
        int c = 0;
        while (c < n_qubits && ((U >> c) & 1u)) ++c;
        r.c = c;
        r.op_begin = int(plan.ops.size());
        for (size_t u = o; u < e; ++u) {
            const CompiledExc &x = exc[op_k[u]];
            OpDev d{};
            d.flip_l = gather_bits(x.flip, U);
            d.occ_l = gather_bits(x.occ, U);
            d.par_l = gather_bits(x.par, U);
            d.par_rest = x.par & ~U;
            d.nb = x.nb;
            int k = 0;
            for (int b = 0; b < r.L; ++b)
                if ((d.flip_l >> b) & 1u) d.pos[k++] = b;
            d.s0 = x.s0;
            d.op = int(u);
            plan.ops.push_back(d);
        }
        r.op_end = int(plan.ops.size());
        plan.runs.push_back(r);
        o = e;
    }
    return plan;
}

}  // namespace uccsd
