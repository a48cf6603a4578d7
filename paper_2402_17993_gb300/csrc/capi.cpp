// C ABI of the UCCSD library (declared in include/uccsd.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/uccsd.h"
#include "jw.hpp"
#include "kernels.cuh"
#include "plan.hpp"
#include "ctx.hpp"

using namespace uccsd;

namespace {


int binom_int(int m, int k) {
    if (k < 0 || k > m) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (m - k + i) / i;
    return int(r);
}

int pair_idx(int p, int q) { return q * (q - 1) / 2 + p; }  // p < q

template <typename R>
struct HamTables {
    std::vector<MixT<R>> mix;
    std::vector<MixO<R>> mixo, d2ao, d2bo;
    std::vector<R> d2bs;
    std::vector<SglT<R>> s1a, s1b;
    std::vector<DblT<R>> d2a, d2b;
    std::vector<R> spec;
};

// Sort the compiled X-mask groups into the class tables of the H-apply.
// Returns false for a group outside the spin-conserving classes.
template <typename R>
bool make_tables(const CompiledH &H, int n_orb, HamTables<R> *T, std::string *err) {
    const int np = n_orb * (n_orb - 1) / 2;
    const int nq = binom_int(n_orb, 4);
    T->mix.assign(size_t(std::max(np, 1)) * std::max(np, 1), MixT<R>{});
    T->s1a.assign(std::max(np, 1), SglT<R>{});
    T->s1b.assign(std::max(np, 1), SglT<R>{});
    T->d2a.assign(std::max(nq, 1), DblT<R>{});
    T->d2b.assign(std::max(nq, 1), DblT<R>{});
    for (auto &v : T->s1a) v.spec = -1;
    for (auto &v : T->s1b) v.spec = -1;
    auto orbs = [](uint32_t m, int *o) {
        int k = 0;
        for (int t = 0; t < 32; ++t)
            if ((m >> t) & 1u) o[k++] = t;
    };
    for (const GroupT<double> &g : H.groups) {
        uint32_t xa = 0, xb = 0, ja = 0, jb = 0;
        for (int k = 0; k < g.nb; ++k) ((g.pos[k] & 1) ? xb : xa) |= 1u << (g.pos[k] >> 1);
        for (int q = 0; q < 2 * n_orb; ++q)
            if ((g.jmask >> q) & 1u) ((q & 1) ? jb : ja) |= 1u << (q >> 1);
        const uint32_t j = ja | (jb << 16);
        const int na = __builtin_popcount(xa), nbv = __builtin_popcount(xb);
        int o[4];
        if (g.nb == 2 && (na == 2 || nbv == 2)) {
            orbs(na ? xa : xb, o);
            SglT<R> &S = (na ? T->s1a : T->s1b)[pair_idx(o[0], o[1])];
            S.lut[0] = R(g.lut[1]);  // source occupies the lower orbital
            S.lut[1] = R(g.lut[2]);  // source occupies the higher orbital
            S.j = j;
            S.spec = g.spec;
        } else if (g.nb == 4 && (na == 4 || nbv == 4)) {
            orbs(na ? xa : xb, o);
            DblT<R> &D = (na ? T->d2a : T->d2b)[binom_int(o[3], 4) + binom_int(o[2], 3) +
                                                binom_int(o[1], 2) + o[0]];
            for (int p = 0; p < 16; ++p) D.lut[p] = R(g.lut[p]);
            D.j = j;
        } else if (g.nb == 4 && na == 2 && nbv == 2) {
            int oa[4], ob[4];
            orbs(xa, oa);
            orbs(xb, ob);
            MixT<R> &M = T->mix[size_t(pair_idx(oa[0], oa[1])) * np + pair_idx(ob[0], ob[1])];
            for (int asel = 0; asel < 2; ++asel)
                for (int bsel = 0; bsel < 2; ++bsel) {
                    const int qa = 2 * oa[asel], qb = 2 * ob[bsel] + 1;  // occupied by the source
                    int pat = 0;
                    for (int k = 0; k < 4; ++k)
                        if (g.pos[k] == qa || g.pos[k] == qb) pat |= 1 << k;
                    M.lut[asel + 2 * bsel] = R(g.lut[pat]);
                }
            M.j = j;
        } else {
            *err = "X-mask group outside the spin-conserving classes";
            return false;
        }
    }
    for (double v : H.spec) T->spec.push_back(R(v));
    if (T->spec.empty()) T->spec.push_back(R(0));
    // ordered view of the mixed groups (target occupies p and j; the source
    // occupies q and b: asel = q > p, bsel = b > j)
    T->mixo.assign(size_t(n_orb) * n_orb * n_orb * n_orb, MixO<R>{});
    for (int p = 0; p < n_orb; ++p)
        for (int q = 0; q < n_orb; ++q)
            for (int jj = 0; jj < n_orb; ++jj)
                for (int b = 0; b < n_orb; ++b) {
                    if (p == q || jj == b) continue;
                    const MixT<R> &M = T->mix[size_t(pair_idx(std::min(p, q), std::max(p, q))) * np +
                                              pair_idx(std::min(jj, b), std::max(jj, b))];
                    MixO<R> &O = T->mixo[((size_t(p) * n_orb + q) * n_orb + jj) * n_orb + b];
                    O.w = M.lut[(q > p ? 1 : 0) + 2 * (b > jj ? 1 : 0)];
                    O.j = M.j;
                }
    // ordered view of the same-spin doubles
    const size_t n4 = size_t(n_orb) * n_orb * n_orb * n_orb;
    for (int spin = 0; spin < 2; ++spin) {
        std::vector<MixO<R>> &dst = spin ? T->d2bo : T->d2ao;
        const std::vector<DblT<R>> &src = spin ? T->d2b : T->d2a;
        dst.assign(n4, MixO<R>{});
        for (int o1 = 0; o1 < n_orb; ++o1)
            for (int o2 = o1 + 1; o2 < n_orb; ++o2)
                for (int v1 = 0; v1 < n_orb; ++v1)
                    for (int v2 = v1 + 1; v2 < n_orb; ++v2) {
                        if (v1 == o1 || v1 == o2 || v2 == o1 || v2 == o2) continue;
                        int q[4] = {o1, o2, v1, v2};
                        std::sort(q, q + 4);
                        const DblT<R> &D = src[binom_int(q[3], 4) + binom_int(q[2], 3) +
                                               binom_int(q[1], 2) + q[0]];
                        int pat = 0;
                        for (int k = 0; k < 4; ++k)
                            if (q[k] == v1 || q[k] == v2) pat |= 1 << k;
                        MixO<R> &O = dst[((size_t(o1) * n_orb + o2) * n_orb + v1) * n_orb + v2];
                        O.w = D.lut[pat];
                        O.j = D.j;
                    }
    }
    // beta doubles by (occupied pair, empty pair) index with the part of the
    // Jordan-Wigner sign that depends on the excitation alone: the group's
    // beta mask is M = L(o1) ^ L(o2) ^ L(v1) ^ L(v2) without the flipped
    // bits (L(v) = bits below v), and the target occupies o1 and o2, so the
    // source's parity under it is popc(target & M) - bit o1 of M - bit o2
    // of M; the H-apply forms the first term from per-lane prefix parities.
    T->d2bs.assign(size_t(std::max(np, 1)) * std::max(np, 1), R(0));
    for (int o1 = 0; o1 < n_orb; ++o1)
        for (int o2 = o1 + 1; o2 < n_orb; ++o2)
            for (int v1 = 0; v1 < n_orb; ++v1)
                for (int v2 = v1 + 1; v2 < n_orb; ++v2) {
                    if (v1 == o1 || v1 == o2 || v2 == o1 || v2 == o2) continue;
                    const uint32_t M = ((1u << o1) - 1u) ^ ((1u << o2) - 1u) ^ ((1u << v1) - 1u) ^
                                       ((1u << v2) - 1u);
                    const R w = T->d2bo[((size_t(o1) * n_orb + o2) * n_orb + v1) * n_orb + v2].w;
                    T->d2bs[size_t(pair_idx(o1, o2)) * np + pair_idx(v1, v2)] =
                        (((M >> o1) ^ (M >> o2)) & 1u) ? -w : w;
                }
    return true;
}

}  // namespace

namespace {

uccsd_status fail(uccsd_ctx *c, uccsd_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

uccsd_status cuda_fail(uccsd_ctx *c, cudaError_t e, const char *what) {
    c->failed = true;
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return UCCSD_ERR_CUDA;
}

void release(uccsd_ctx *c, const std::string &name) {
    auto it = c->mem.find(name);
    if (it == c->mem.end()) return;
    cudaFree(it->second.first);
    c->bytes -= it->second.second;
    c->mem.erase(it);
}

// A named device buffer of at least `bytes`; contents are undefined.  A
// buffer only grows (cudaFree waits for the whole device, so a context that
// is refilled with a problem of the same shape class frees nothing); on
// growth it takes 1/8 headroom when the budget allows.
uccsd_status dalloc(uccsd_ctx *c, const std::string &name, size_t bytes, void **out) {
    auto it = c->mem.find(name);
    if (it != c->mem.end() && it->second.second >= bytes) {
        *out = it->second.first;
        return UCCSD_OK;
    }
    const bool grow = it != c->mem.end();
    release(c, name);
    bytes = std::max<size_t>(bytes, 16);
    if (c->budget && c->bytes + bytes > c->budget)
        return fail(c, UCCSD_ERR_BUDGET, "device footprint of '" + name + "' exceeds the HBM budget");
    if (grow && (!c->budget || c->bytes + bytes + bytes / 8 <= c->budget)) bytes += bytes / 8;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, UCCSD_ERR_OOM, "cudaMalloc of '" + name + "' failed: " + cudaGetErrorString(e));
    }
    c->mem[name] = {p, bytes};
    c->bytes += bytes;
    *out = p;
    return UCCSD_OK;
}

void *dptr(uccsd_ctx *c, const std::string &name) {
    auto it = c->mem.find(name);
    return it == c->mem.end() ? nullptr : it->second.first;
}

// Host wait for the set-up transfers when they run on the context's own
// stream; none when they are ordered on a caller stream.
cudaError_t setup_sync(uccsd_ctx *c) {
    return c->setup_async ? cudaSuccess : cudaStreamSynchronize(c->setup);
}

// Copy `nb` host bytes into the pinned staging area; *out is the staged copy.
// The area is reused from its start once the copies staged earlier (all on
// the context's own stream, before the last recorded stage_ev) are done.
uccsd_status stage_bytes(uccsd_ctx *c, const void *src, size_t nb, const void **out) {
    const size_t need = (nb + 255) & ~size_t(255);
    cudaError_t e = cudaSuccess;
    if (c->stage_off + need > c->stage_cap) {
        if (c->stage_off > 0 && (e = cudaEventSynchronize(c->stage_ev)) != cudaSuccess)
            return cuda_fail(c, e, "staging wait");
        c->stage_off = 0;
        if (need > c->stage_cap) {
            if (c->stage) cudaFreeHost(c->stage);
            c->stage = nullptr;
            c->stage_cap = 0;
            const size_t cap = std::max(need, size_t(1) << 20);
            if ((e = cudaHostAlloc(reinterpret_cast<void **>(&c->stage), cap, cudaHostAllocDefault)) !=
                cudaSuccess) {
                cudaGetLastError();
                c->stage = nullptr;
                return fail(c, UCCSD_ERR_OOM, "pinned staging allocation failed");
            }
            c->stage_cap = cap;
        }
    }
    std::memcpy(c->stage + c->stage_off, src, nb);
    *out = c->stage + c->stage_off;
    c->stage_off += need;
    return UCCSD_OK;
}

template <typename T>
uccsd_status upload(uccsd_ctx *c, const std::string &name, const std::vector<T> &v, T **out) {
    void *p = nullptr;
    uccsd_status st = dalloc(c, name, sizeof(T) * std::max<size_t>(v.size(), 1), &p);
    if (st) return st;
    if (!v.empty()) {
        const size_t nb = sizeof(T) * v.size();
        cudaError_t e;
        if (c->setup_async) {
            // the copy runs on the context's own stream and the caller's
            // stream waits for it: the staging event is only ever recorded
            // on a stream that no other thread captures or shares
            const void *src = nullptr;
            if ((st = stage_bytes(c, v.data(), nb, &src))) return st;
            e = cudaMemcpyAsync(p, src, nb, cudaMemcpyHostToDevice, c->own_setup);
            if (e == cudaSuccess) e = cudaEventRecord(c->stage_ev, c->own_setup);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->setup, c->stage_ev, 0);
        } else {
            e = cudaMemcpyAsync(p, v.data(), nb, cudaMemcpyHostToDevice, c->setup);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->setup);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "upload");
    }
    *out = static_cast<T *>(p);
    return UCCSD_OK;
}

// Fixed-point form of the diagonal: unit 2^-k with k chosen so that every
// partial sum of |c0| + sum |a| + sum |b| (times 2 for the shift) fits in
// 62 bits.  Quantisation error <= 2^-(k+1) per term.
void make_fixed_point(uccsd_ctx *c) {
    const CompiledH &H = c->H;
    double bound = std::fabs(H.c0);
    for (double v : H.diag_a) bound += std::fabs(v);
    for (double v : H.diag_b) bound += std::fabs(v);
    bound = 2.0 * bound + 1.0;
    int k = 61 - int(std::ceil(std::log2(bound)));
    k = std::max(0, std::min(k, 60));
    double scale = std::ldexp(1.0, k);
    c->diag_unit = std::ldexp(1.0, -k);
    c->diag_qa.resize(H.diag_a.size());
    c->diag_qb.resize(H.diag_b.size());
    for (size_t i = 0; i < H.diag_a.size(); ++i) c->diag_qa[i] = std::llround(H.diag_a[i] * scale);
    for (size_t i = 0; i < H.diag_b.size(); ++i) c->diag_qb[i] = std::llround(H.diag_b[i] * scale);
}

// Diagonal constant after the shift, in fixed point.
long long shifted_q0(const uccsd_ctx *c) {
    return std::llround((c->H.c0 - c->shift) / c->diag_unit);
}

template <typename R>
uccsd_status upload_ham(uccsd_ctx *c, DevHam<R> *dh, const char *tag) {
    HamTables<R> T;
    std::string err;
    if (!make_tables<R>(c->H, c->n_orb, &T, &err)) return fail(c, UCCSD_ERR_ARG, err);
    std::string t(tag);
    c->spec_s1a.resize(T.s1a.size());
    c->spec_s1b.resize(T.s1b.size());
    for (size_t i = 0; i < T.s1a.size(); ++i) c->spec_s1a[i] = T.s1a[i].spec;
    for (size_t i = 0; i < T.s1b.size(); ++i) c->spec_s1b[i] = T.s1b[i].spec;
    MixT<R> *mx;
    MixO<R> *mo, *oa, *ob;
    R *bs;
    SglT<R> *sa, *sb;
    DblT<R> *da, *db;
    R *sp;
    long long *qa, *qb;
    uccsd_status st;
    if ((st = upload(c, t + "mix", T.mix, &mx))) return st;
    if ((st = upload(c, t + "mixo", T.mixo, &mo))) return st;
    if ((st = upload(c, t + "d2ao", T.d2ao, &oa))) return st;
    if ((st = upload(c, t + "d2bo", T.d2bo, &ob))) return st;
    if ((st = upload(c, t + "d2bs", T.d2bs, &bs))) return st;
    if ((st = upload(c, t + "s1a", T.s1a, &sa))) return st;
    if ((st = upload(c, t + "s1b", T.s1b, &sb))) return st;
    if ((st = upload(c, t + "d2a", T.d2a, &da))) return st;
    if ((st = upload(c, t + "d2b", T.d2b, &db))) return st;
    if ((st = upload(c, t + "spec", T.spec, &sp))) return st;
    if ((st = upload(c, "diag_qa", c->diag_qa, &qa))) return st;
    if ((st = upload(c, "diag_qb", c->diag_qb, &qb))) return st;
    dh->mix = mx;
    dh->mixo = mo;
    dh->d2ao = oa;
    dh->d2bo = ob;
    dh->d2bs = bs;
    dh->s1a = sa;
    dh->s1b = sb;
    dh->d2a = da;
    dh->d2b = db;
    dh->spec = sp;
    dh->diag_qa = qa;
    dh->diag_qb = qb;
    dh->diag_q0 = shifted_q0(c);
    dh->diag_unit = c->diag_unit;
    dh->has_diag = c->H.has_diag ? 1 : 0;
    dh->n = c->n;
    dh->n_orb = c->n_orb;
    dh->n_pairs = c->n_orb * (c->n_orb - 1) / 2;
    return UCCSD_OK;
}

// Combinatorial rank tables (shared by the sweeps and the H-apply) and the
// string -> global bit deposits of the H-apply's row/column layout (alpha
// string bit t = qubit 2t, beta string bit t = qubit 2t + 1).
uccsd_status upload_tile_tables(uccsd_ctx *c) {
    // the tables do not depend on the problem: built once per process
    static std::once_flag once;
    static std::vector<uint16_t> combos, ranks;
    static std::vector<int32_t> coffs;
    std::call_once(once, [] { build_comb_tables(&combos, &ranks, &coffs); });
    uint16_t *p5;
    int32_t *p2;
    uint32_t *p4;
    uccsd_status st;
    if ((st = upload(c, "combos", combos, &p5))) return st;
    c->comb_combos = p5;
    if ((st = upload(c, "ranks", ranks, &p5))) return st;
    c->comb_ranks = p5;
    if ((st = upload(c, "comb_offs", coffs, &p2))) return st;
    c->comb_offs = p2;
    c->comb_offs_host = coffs;
    const int no = c->n_orb;
    std::vector<uint32_t> spread(size_t(2) << no);
    for (uint32_t s = 0; s < (1u << no); ++s) {
        uint32_t a = 0, b = 0;
        for (int k = 0; k < no; ++k)
            if ((s >> k) & 1u) {
                a |= 1u << (2 * k);
                b |= 1u << (2 * k + 1);
            }
        spread[s] = a;
        spread[(size_t(1) << no) + s] = b;
    }
    if ((st = upload(c, "hspread", spread, &p4))) return st;
    c->hsec.aspread = p4;
    c->hsec.bspread = p4 + (size_t(1) << no);
    std::vector<int32_t> bn(16 * 5);
    for (int t = 0; t < 16; ++t)
        for (int k = 0; k <= 4; ++k) bn[t * 5 + k] = binom_int(t, k);
    if ((st = upload(c, "binom", bn, &p2))) return st;
    c->hsec.binom = p2;
    c->hsec.brank = c->comb_ranks + ((size_t(1) << no) - 1);
    return UCCSD_OK;
}

// Row/column layout of the sector for the reference's electron counts and
// the state addressing of the context's layout.
// Beta-spectator sums of the pair groups per column of the reference's
// beta strings (see DevHam::bspec_a / bspec_b), summed in FP64 and rounded
// once to R.
template <typename R>
uccsd_status upload_spectator_tables(uccsd_ctx *c, DevHam<R> *dh, const char *tag) {
    const int no = c->n_orb;
    std::vector<uint32_t> bstr;
    for (uint32_t sv = 0; sv < (1u << no); ++sv)
        if (__builtin_popcount(sv) == c->n_beta) bstr.push_back(sv);
    const size_t Db = bstr.size();
    const int np = no * (no - 1) / 2;
    const std::vector<double> &spec = c->H.spec;
    auto row_sum = [&](int spec_row, int pat, uint32_t occ) {
        double v = 0.0;
        for (uint32_t w = occ; w; w &= w - 1u)
            v += spec[size_t(spec_row + 2 * __builtin_ctz(w) + 1) * 4 + pat];
        return v;
    };
    std::vector<R> ta(size_t(2) * std::max(np, 1) * std::max<size_t>(Db, 1), R(0));
    for (int pa = 0; pa < np; ++pa) {
        const int sr = pa < int(c->spec_s1a.size()) ? c->spec_s1a[pa] : -1;
        if (sr < 0) continue;
        for (int sel = 0; sel < 2; ++sel)
            for (size_t col = 0; col < Db; ++col)
                ta[(size_t(pa) * 2 + sel) * Db + col] = R(row_sum(sr, sel ? 2 : 1, bstr[col]));
    }
    const int ns = c->n_beta * (no - c->n_beta);
    std::vector<R> tb(size_t(std::max(ns, 1)) * std::max<size_t>(Db, 1), R(0));
    for (size_t col = 0; col < Db; ++col) {
        const uint32_t sb = bstr[col];
        int k = 0;
        for (int j = 0; j < no; ++j) {
            if (!((sb >> j) & 1u)) continue;
            for (int bb = 0; bb < no; ++bb) {
                if ((sb >> bb) & 1u) continue;
                const int pb = pair_idx(std::min(j, bb), std::max(j, bb));
                const int sr = pb < int(c->spec_s1b.size()) ? c->spec_s1b[pb] : -1;
                const uint32_t yb = sb ^ (1u << j) ^ (1u << bb);
                if (sr >= 0) tb[size_t(k) * Db + col] = R(row_sum(sr, bb > j ? 2 : 1, yb & ~(1u << bb)));
                ++k;
            }
        }
    }
    // beta-qubit part of the diagonal's fixed-point form per column (beta
    // orbital j is qubit 2j + 1)
    std::vector<long long> dc(std::max<size_t>(Db, 1), 0);
    const int n = c->n;
    for (size_t col = 0; col < Db; ++col) {
        long long q = 0;
        for (uint32_t w = bstr[col]; w; w &= w - 1u) {
            const int r = 2 * __builtin_ctz(w) + 1;
            q += c->diag_qa[r];
            for (uint32_t w2 = w & (w - 1u); w2; w2 &= w2 - 1u)
                q += c->diag_qb[size_t(r) * n + 2 * __builtin_ctz(w2) + 1];
        }
        dc[col] = q;
    }
    std::string t(tag);
    R *pa_, *pb_;
    long long *dc_;
    uccsd_status st;
    if ((st = upload(c, t + "bspec_a", ta, &pa_))) return st;
    if ((st = upload(c, t + "bspec_b", tb, &pb_))) return st;
    if ((st = upload(c, t + "diag_col", dc, &dc_))) return st;
    dh->bspec_a = pa_;
    dh->bspec_b = pb_;
    dh->diag_col = dc_;
    return UCCSD_OK;
}

// Whether state addressing tables are the sector order's (where the plans'
// entry maps apply).
bool sector_order(const uccsd_ctx *c, const uint32_t *aoff, const uint32_t *boff) {
    return aoff && aoff == c->sec_aoff && boff == c->sec_boff;
}

// Optimiser records in one pinned, mapped block allocated at the first
// uccsd_opt_init of the process: the optimiser kernel writes a context's
// meta words and energy history there, and uccsd_opt_history reads them from
// host memory after the context's stream is done, without a copy on any
// stream (a copy could queue behind other streams' work on a shared hardware
// queue, such as solves held by gates, and wait for it).
constexpr int kOptRecDoubles = 1024;  // 2 doubles of meta ints, then up to 1022 energies
constexpr int kOptRecs = 1024;
std::mutex g_opt_mu;
double *g_opt_block = nullptr;
std::vector<int> *g_opt_free = nullptr;  // never destroyed (no CUDA calls at exit)

double *opt_rec_take() {
    std::lock_guard<std::mutex> lk(g_opt_mu);
    if (!g_opt_block) {
        if (g_opt_free) return nullptr;  // the allocation failed once
        g_opt_free = new std::vector<int>();
        void *p = nullptr;
        if (cudaHostAlloc(&p, sizeof(double) * kOptRecDoubles * kOptRecs,
                          cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_opt_block = static_cast<double *>(p);
        for (int i = kOptRecs - 1; i >= 0; --i) g_opt_free->push_back(i);
    }
    if (g_opt_free->empty()) return nullptr;
    const int i = g_opt_free->back();
    g_opt_free->pop_back();
    return g_opt_block + size_t(i) * kOptRecDoubles;
}

void opt_rec_give(double *r) {
    if (!r) return;
    std::lock_guard<std::mutex> lk(g_opt_mu);
    g_opt_free->push_back(int((r - g_opt_block) / kOptRecDoubles));
}

int *opt_meta_ptr(uccsd_ctx *c) {
    return c->opt_rec_dev ? reinterpret_cast<int *>(c->opt_rec_dev) : opt_meta_ptr(c);
}
double *opt_hist_ptr(uccsd_ctx *c) {
    return c->opt_rec_dev ? c->opt_rec_dev + 2 : opt_hist_ptr(c);
}

// The entry maps of a sweep plan (build_entry_map, plan.cpp) on the device.
// No map (all emap_base = -1) when it would hold
// more than kMaxMapEntries entries (2 GB), or take more than half of a
// context's HBM budget (the state vectors come later).  26 qubits: 1.2 GB
// for both plans, evaluation 27.9 -> 26.3 ms.
constexpr size_t kMaxMapEntries = size_t(512) << 20;
uccsd_status attach_entry_map(uccsd_ctx *c, SweepPlan *pl, const std::string &name,
                              const uint32_t **out) {
    *out = nullptr;
    size_t total = 0;
    for (CRunDev &r : pl->runs) {
        r.emap_base = -1;
        total += size_t(r.n_tiles) * size_t(r.max_entries);
    }
    if (total == 0 || total > kMaxMapEntries) return UCCSD_OK;
    if (c->budget && c->bytes + sizeof(uint32_t) * total > c->budget / 2) return UCCSD_OK;
    const std::vector<uint32_t> map = build_entry_map(c->n, c->n_alpha, c->n_beta, pl);
    uint32_t *p;
    uccsd_status st = upload(c, name, map, &p);
    if (st) {
        for (CRunDev &r : pl->runs) r.emap_base = -1;
        return st;
    }
    *out = p;
    return UCCSD_OK;
}

// happly_mixed_order per (n_orb, n_beta), computed once per process.
const std::vector<uint8_t> &mixed_order(int n_orb, int n_beta) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, std::vector<uint8_t>> *cache =
        new std::map<std::pair<int, int>, std::vector<uint8_t>>();
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache->find({n_orb, n_beta});
    if (it == cache->end()) it = cache->emplace(std::make_pair(n_orb, n_beta), happly_mixed_order(n_orb, n_beta)).first;
    return it->second;
}

uccsd_status set_row_layout(uccsd_ctx *c) {
    const int no = c->n_orb;
    const size_t base = (size_t(1) << no) - 1;
    c->hsec.astr = c->comb_combos + base + c->comb_offs_host[no * 17 + c->n_alpha];
    c->hsec.bstr = c->comb_combos + base + c->comb_offs_host[no * 17 + c->n_beta];
    c->hsec.Da = binom_int(no, c->n_alpha);
    c->hsec.Db = binom_int(no, c->n_beta);
    c->hsec.colblock = std::min(c->hsec.Db, kHColBlock);
    c->hsec.ncb = (c->hsec.Db + c->hsec.colblock - 1) / c->hsec.colblock;
    c->hsec.n_alpha = c->n_alpha;
    c->hsec.n_beta = c->n_beta;
    c->hsec.aoff = c->hsec.aspread;
    c->hsec.boff = c->hsec.bspread;
    {
        // beta single excitations of every column (layout independent)
        std::vector<uint32_t> bstr_h, rank_h(size_t(1) << no, 0u);
        for (uint32_t sv = 0; sv < (1u << no); ++sv)
            if (__builtin_popcount(sv) == c->n_beta) {
                rank_h[sv] = uint32_t(bstr_h.size());
                bstr_h.push_back(sv);
            }
        const int Db = int(bstr_h.size());
        const int ns = c->n_beta * (no - c->n_beta);
        std::vector<uint32_t> tab(size_t(2) * std::max(ns, 1) * std::max(Db, 1), 0u);
        std::vector<uint32_t> mix(size_t(std::max(ns, 1)) * std::max(Db, 1), 0u);
        for (int col = 0; col < Db; ++col) {
            const uint32_t sb = bstr_h[col];
            int k = 0;
            for (int j = 0; j < no; ++j) {
                if (!((sb >> j) & 1u)) continue;
                for (int bb = 0; bb < no; ++bb) {
                    if ((sb >> bb) & 1u) continue;
                    const uint32_t yb = sb ^ (1u << j) ^ (1u << bb);
                    const size_t at = 2 * (size_t(k) * Db + col);
                    const int lo = std::min(j, bb), hi = std::max(j, bb);
                    tab[at] = rank_h[yb] | (uint32_t(j * no + bb) << 16);
                    // the column's part of the single's sign: parities of the
                    // occupied beta orbitals below j and below b, and b > j
                    const uint32_t cs = uint32_t(__builtin_popcount(sb & ((1u << j) - 1u)) +
                                                 __builtin_popcount(sb & ((1u << bb) - 1u)) + (bb > j)) & 1u;
                    tab[at + 1] = cs | (uint32_t(2 * pair_idx(lo, hi) + (bb > j)) << 16);
                    // occupied beta orbitals strictly between j and b
                    const uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
                    const uint32_t pi = uint32_t(__builtin_popcount(sb & between) & 1);
                    mix[size_t(k) * Db + col] = rank_h[yb] | (uint32_t(j * no + bb + no * no * pi) << 16);
                    ++k;
                }
            }
        }
        if (c->prec && happly_cols_per_thread(c->hsec) == 1) {
            // FP32 at one column per thread: the mixed groups take each
            // column's singles in the order that spreads a wavefront's
            // 16-byte loads over the bank groups
            const std::vector<uint8_t> &ord = mixed_order(no, c->n_beta);
            std::vector<uint32_t> nat(mix);
            for (size_t t = 0; t < size_t(ns); ++t)
                for (size_t col = 0; col < size_t(Db); ++col)
                    mix[t * Db + col] = nat[size_t(ord[t * Db + col]) * Db + col];
        }
        uint32_t *p4, *pm;
        uccsd_status st = upload(c, "bsing", tab, &p4);
        if (st) return st;
        if ((st = upload(c, "bmix", mix, &pm))) return st;
        c->hsec.bsing = reinterpret_cast<const uint2 *>(p4);
        c->hsec.bmix = pm;
        c->hsec.n_bs = ns;
        // alpha singles per H-apply phase: up to 4 while their staged source
        // rows take at most 64 KiB (FP32) or 24 KiB (FP64) of shared memory.
        // Measured at 26 qubits (1716 columns): FP32 four per phase against one,
        // 13.4 against 18.9 ms; FP64 one per phase, since two cost occupancy.
        const size_t row = size_t(Db) * (c->prec ? 8 : 16);  // one staged source row
        const size_t cap = size_t(c->prec ? 64 : 24) << 10;
        c->hsec.ag = 1;
        while (c->hsec.ag < 4 && size_t(2 * c->hsec.ag) * row <= cap) c->hsec.ag *= 2;
    }
    c->hsec_full = c->hsec;
    {
        uccsd_status st = c->prec ? upload_spectator_tables<float>(c, &c->hf32, "h32_")
                                  : upload_spectator_tables<double>(c, &c->hf64, "h64_");
        if (st) return st;
    }
    const uint32_t hfa = uint32_t((1u << c->n_alpha) - 1u), hfb = uint32_t((1u << c->n_beta) - 1u);
    c->hf_addr = c->hf;
    {
        // sector addressing: rank of a string among the n_orb-bit strings of
        // its popcount, in ascending order (the order of astr / bstr).  The
        // sector layout stores states this way; the full layout uses it for
        // the sweeps' hand-over between runs.
        std::vector<uint32_t> off(size_t(2) << no, 0u);
        std::vector<int> cnt(no + 2, 0);
        for (uint32_t sv = 0; sv < (1u << no); ++sv) {
            const int pc = __builtin_popcount(sv);
            const uint32_t rank = uint32_t(cnt[pc]++);
            if (pc == c->n_alpha) off[sv] = rank * uint32_t(c->hsec.Db);
            if (pc == c->n_beta) off[(size_t(1) << no) + sv] = rank;
        }
        uint32_t *p4;
        uccsd_status st = upload(c, "hoff", off, &p4);
        if (st) return st;
        c->sec_aoff = p4;
        c->sec_boff = p4 + (size_t(1) << no);
        c->hsec_sec = c->hsec;
        c->hsec_sec.aoff = c->sec_aoff;
        c->hsec_sec.boff = c->sec_boff;
        c->hf_sec = off[hfa] + off[(size_t(1) << no) + hfb];
        if (c->layout == UCCSD_LAYOUT_SECTOR) {
            c->hsec.aoff = c->sec_aoff;
            c->hsec.boff = c->sec_boff;
            c->hf_addr = off[hfa] + off[(size_t(1) << no) + hfb];
        }
    }
    if (c->layout == UCCSD_LAYOUT_SCBK) {
        // tapered Bravyi-Kitaev positions of the sector determinants
        std::vector<uint32_t> ta, tb;
        scbk_addresses(no, &ta, &tb);
        std::vector<uint32_t> off(ta);
        off.insert(off.end(), tb.begin(), tb.end());
        uint32_t *p4;
        uccsd_status st = upload(c, "scbkoff", off, &p4);
        if (st) return st;
        c->hsec.aoff = p4;
        c->hsec.boff = p4 + (size_t(1) << no);
        c->hf_addr = ta[hfa] + tb[hfb];
    }
    return UCCSD_OK;
}

// Amplitudes per slot: 2^n in the full layout, Da * Db in the sector layout.
size_t state_elems(const uccsd_ctx *c) {
    if (c->layout == UCCSD_LAYOUT_SECTOR) return size_t(c->hsec.Da) * size_t(c->hsec.Db);
    return size_t(1) << (c->layout == UCCSD_LAYOUT_SCBK ? c->n - 2 : c->n);
}
size_t amp_bytes(const uccsd_ctx *c) { return c->prec ? 8 : 16; }
int n_tiles_h(const uccsd_ctx *c) { return c->hsec.Da * c->hsec.ncb; }
int n_tiles_a(const uccsd_ctx *c) { return c->adj.max_tiles; }

// Per-slot buffers sized for c->B slots.
uccsd_status alloc_slots(uccsd_ctx *c) {
    if (!c->have_exc) return UCCSD_OK;
    void *p;
    uccsd_status st;
    const size_t B = c->B;
    const size_t n_ops = std::max<size_t>(c->op_k.size(), 1);
    if ((st = dalloc(c, "psi", B * state_elems(c) * amp_bytes(c), &p))) return st;
    // the sweeps touch only electron-sector amplitudes; the rest stays zero
    cudaError_t e0 = cudaMemsetAsync(p, 0, B * state_elems(c) * amp_bytes(c), c->setup);
    if (e0 != cudaSuccess) return cuda_fail(c, e0, "memset");
    if ((st = dalloc(c, "sig", B * state_elems(c) * amp_bytes(c), &p))) return st;
    // sigma is written only inside the electron sector; the rest stays zero
    cudaError_t e = cudaMemsetAsync(p, 0, B * state_elems(c) * amp_bytes(c), c->setup);
    if (e == cudaSuccess) e = setup_sync(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset");
    // Full layout, adjoint of several runs: each run hands phi and lambda to
    // the next in the compact sector order instead of scattering them into
    // the 2^n vectors and gathering them back (every run writes all sector
    // entries of its tiles before the next one reads them, so no clearing).
    // The forward's runs hand the state on the same way (the forward is done
    // before the adjoint starts, so the two share the first array).
    const bool vec = c->layout != UCCSD_LAYOUT_SECTOR;  // a basis vector per slot (2^n or 2^(n-2))
    c->adj_compact = vec && c->adj.runs.size() > 1;
    c->fwd_compact = vec && c->fwd.runs.size() > 1;
    const size_t D = size_t(c->hsec.Da) * size_t(c->hsec.Db);
    if (c->adj_compact || c->fwd_compact) {
        if ((st = dalloc(c, "phic", B * D * amp_bytes(c), &p))) return st;
        if (c->adj_compact && (st = dalloc(c, "lamc", B * D * amp_bytes(c), &p))) return st;
    }
    // Full layout, energy and gradient: the forward leaves psi, and the
    // H-apply sigma, in the compact sector order, where the H-apply and the
    // adjoint read them (nothing reads the 2^n vectors after a gradient
    // call; energy-only calls keep psi in the 2^n vector for uccsd_get_state).
    if (vec) {
        if ((st = dalloc(c, "psic", B * D * amp_bytes(c), &p))) return st;
        if ((st = dalloc(c, "sigc", B * D * amp_bytes(c), &p))) return st;
    }
    if ((st = dalloc(c, "cs", B * n_ops * amp_bytes(c), &p))) return st;
    if ((st = dalloc(c, "theta", B * std::max(c->K, 1) * sizeof(double), &p))) return st;
    if ((st = dalloc(c, "E", B * sizeof(double), &p))) return st;
    if ((st = dalloc(c, "grad", B * std::max(c->K, 1) * sizeof(double), &p))) return st;
    if ((st = dalloc(c, "Epart", 2 * B * n_tiles_h(c) * sizeof(double), &p))) return st;
    if ((st = dalloc(c, "gpart", B * n_ops * n_tiles_a(c) * sizeof(double), &p))) return st;
    return UCCSD_OK;
}

bool finite_all(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

uccsd_status check_hamiltonian_input(uccsd_ctx *c, int n_orb, const double *h, const double *eri,
                                     double e_core) {
    if (n_orb < 1 || n_orb > 15) return fail(c, UCCSD_ERR_ARG, "n_orb must be in [1, 15]");
    if (!h || !eri) return fail(c, UCCSD_ERR_ARG, "null integral pointer");
    const size_t no = n_orb;
    if (!finite_all(h, no * no) || !finite_all(eri, no * no * no * no) || !std::isfinite(e_core))
        return fail(c, UCCSD_ERR_ARG, "non-finite integral");
    for (size_t p = 0; p < no; ++p)
        for (size_t q = 0; q < no; ++q)
            if (std::fabs(h[p * no + q] - h[q * no + p]) > 1e-12)
                return fail(c, UCCSD_ERR_ARG, "h is not symmetric");
    auto E = [&](size_t p, size_t q, size_t r, size_t s) { return eri[((p * no + q) * no + r) * no + s]; };
    for (size_t p = 0; p < no; ++p)
        for (size_t q = 0; q < no; ++q)
            for (size_t r = 0; r < no; ++r)
                for (size_t s = 0; s < no; ++s) {
                    double v = E(p, q, r, s);
                    if (std::fabs(v - E(q, p, r, s)) > 1e-12 || std::fabs(v - E(p, q, s, r)) > 1e-12 ||
                        std::fabs(v - E(r, s, p, q)) > 1e-12)
                        return fail(c, UCCSD_ERR_ARG, "eri lacks the 8-fold permutational symmetry");
                }
    return UCCSD_OK;
}

// Event marker between kernel families (profiling only).
struct Marks {
    uccsd_ctx *c;
    cudaStream_t s;
    std::vector<std::pair<int, int>> spans;  // (family, event index of its start)
    int next = 0;
    void begin(int fam) {
        if (!c->profiling) return;
        if (next >= int(c->events.size())) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->events.push_back(e);
        }
        cudaEventRecord(c->events[next], s);
        spans.push_back({fam, next});
        ++next;
    }
    void finish() {
        if (!c->profiling) return;
        begin(-1);
        cudaEventSynchronize(c->events[next - 1]);
        for (size_t i = 0; i + 1 < spans.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->events[spans[i].second], c->events[spans[i + 1].second]);
            c->prof.ms[spans[i].first] += ms;
        }
        c->prof.calls++;
    }
};

template <typename R>
uccsd_status run_eval(uccsd_ctx *c, int B, const double *theta, int on_dev, double *E, double *grad,
                      cudaStream_t stream) {
    const size_t N = state_elems(c);
    LaunchCfg cfg;
    cfg.n = c->n;
    cfg.N = N;
    cfg.B = B;
    cfg.n_ops = int(c->op_k.size());
    cfg.stream = stream;
    const int K = c->K;
    cudaError_t e;
    double *d_theta = static_cast<double *>(dptr(c, "theta"));
    const double *th = theta;
    if (!on_dev) {
        e = cudaMemcpyAsync(d_theta, theta, sizeof(double) * B * K, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "theta upload");
        th = d_theta;
    }
    void *psi = dptr(c, "psi"), *sig = dptr(c, "sig"), *cs = dptr(c, "cs");
    double *Epart = static_cast<double *>(dptr(c, "Epart"));
    double *gpart = static_cast<double *>(dptr(c, "gpart"));
    const int32_t *d_op_k = static_cast<const int32_t *>(dptr(c, "op_k"));
    const double *d_op_scale = static_cast<const double *>(dptr(c, "op_scale"));
    Marks mk{c, stream};
    if (cfg.n_ops > 0) {
        mk.begin(UCCSD_K_CS);
        if ((e = launch_cs<R>(cfg, th, K, d_op_k, d_op_scale, cs)) != cudaSuccess)
            return cuda_fail(c, e, "cs kernel");
        ++c->launches;
        c->prof.launches[UCCSD_K_CS]++;
    }
    const COpDev *fops = static_cast<const COpDev *>(dptr(c, "fwd_ops"));
    mk.begin(UCCSD_K_FORWARD);
    const size_t Dsec = size_t(c->hsec.Da) * size_t(c->hsec.Db);
    void *phic = (c->fwd_compact || c->adj_compact) ? dptr(c, "phic") : nullptr;
    // full layout with a gradient: psi and sigma stay in the compact sector
    // order from the forward's last run to the adjoint's first
    const bool compact_path = c->layout != UCCSD_LAYOUT_SECTOR && grad;
    void *psi_h = compact_path ? dptr(c, "psic") : psi;  // psi as the H-apply reads it
    void *sig_h = compact_path ? dptr(c, "sigc") : sig;
    const int Rf = int(c->fwd.runs.size());
    for (int r = 0; r < Rf; ++r) {
        // full layout, several runs: the runs hand the state to each other in
        // the compact sector order; the last one writes psi
        LaunchCfg fcfg = cfg;
        SweepArgs in = c->fwd_args;
        void *psi_in = psi;
        if (c->fwd_compact && r > 0) {
            psi_in = phic;
            fcfg.N = Dsec;
            in.aoff = c->sec_aoff;
            in.boff = c->sec_boff;
        }
        SweepOut out;
        if ((c->fwd_compact && r + 1 < Rf) || (compact_path && r + 1 == Rf)) {
            out.phi = r + 1 < Rf ? phic : psi_h;
            out.N = Dsec;
            out.aoff = c->sec_aoff;
            out.boff = c->sec_boff;
        } else {
            out.phi = psi;
            out.N = N;
            out.aoff = c->fwd_args.aoff;
            out.boff = c->fwd_args.boff;
        }
        in.emap = sector_order(c, in.aoff, in.boff) ? c->fwd_emap : nullptr;
        out.emap = sector_order(c, out.aoff, out.boff) ? c->fwd_emap : nullptr;
        if ((e = launch_forward_sweep<R>(fcfg, psi_in, c->fwd.runs[r], fops, cs, in, r == 0 ? 1 : 0,
                                         c->hf_addr, out)) != cudaSuccess)
            return cuda_fail(c, e, "forward kernel");
        ++c->launches;
        c->prof.launches[UCCSD_K_FORWARD]++;
    }
    if (c->fwd.runs.empty()) {
        LaunchCfg hcfg = cfg;
        if (compact_path) {  // the compact array holds the last call's state: clear it first
            hcfg.N = Dsec;
            e = cudaMemsetAsync(psi_h, 0, size_t(B) * Dsec * amp_bytes(c), stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "state clear");
        }
        if ((e = launch_set_hf<R>(hcfg, psi_h, compact_path ? c->hf_sec : c->hf_addr)) != cudaSuccess)
            return cuda_fail(c, e, "hf kernel");
        ++c->launches;
        c->prof.launches[UCCSD_K_FORWARD]++;
    }
    const DevHam<R> &H = *reinterpret_cast<const DevHam<R> *>(sizeof(R) == 4 ? (const void *)&c->hf32
                                                                             : (const void *)&c->hf64);
    mk.begin(UCCSD_K_HAPPLY);
    {
        LaunchCfg hcfg = cfg;
        if (compact_path) hcfg.N = Dsec;
        if ((e = launch_happly<R>(hcfg, psi_h, sig_h, c->LH, H, compact_path ? c->hsec_sec : c->hsec,
                                  Epart, grad ? kHApplyStoreSigma : 0)) != cudaSuccess)
            return cuda_fail(c, e, "H-apply kernel");
    }
    ++c->launches;
    c->prof.launches[UCCSD_K_HAPPLY]++;
    if (grad) {
        const COpDev *aops = static_cast<const COpDev *>(dptr(c, "adj_ops"));
        mk.begin(UCCSD_K_ADJOINT);
        // the last run (first in the schedule) leaves phi and lambda nowhere:
        // nothing reads them after the gradient
        const int R_ = int(c->adj.runs.size());
        void *lamc = c->adj_compact ? dptr(c, "lamc") : nullptr;
        for (int r = R_ - 1; r >= 0; --r) {
            LaunchCfg acfg = cfg;
            SweepArgs in = c->adj_args;
            void *phi_in = psi_h, *lam_in = sig_h;
            if (c->adj_compact && r != R_ - 1) {  // read what the previous run handed over
                phi_in = phic;
                lam_in = lamc;
            }
            if (compact_path) {
                acfg.N = Dsec;
                in.aoff = c->sec_aoff;
                in.boff = c->sec_boff;
            }
            SweepOut out;
            if (r > 0) {
                if (c->adj_compact) {
                    out.phi = phic;
                    out.lam = lamc;
                    out.N = Dsec;
                    out.aoff = c->sec_aoff;
                    out.boff = c->sec_boff;
                } else {  // in place
                    out.phi = phi_in;
                    out.lam = lam_in;
                    out.N = acfg.N;
                    out.aoff = in.aoff;
                    out.boff = in.boff;
                }
            }
            in.emap = sector_order(c, in.aoff, in.boff) ? c->adj_emap : nullptr;
            out.emap = sector_order(c, out.aoff, out.boff) ? c->adj_emap : nullptr;
            if ((e = launch_adjoint_sweep<R>(acfg, phi_in, lam_in, c->adj.runs[r], aops, cs, in,
                                             gpart, n_tiles_a(c), out)) != cudaSuccess)
                return cuda_fail(c, e, "adjoint kernel");
            ++c->launches;
            c->prof.launches[UCCSD_K_ADJOINT]++;
        }
    }
    mk.begin(UCCSD_K_REDUCE);
    double *dE = on_dev ? E : static_cast<double *>(dptr(c, "E"));
    double *dG = grad ? (on_dev ? grad : static_cast<double *>(dptr(c, "grad"))) : nullptr;
    if ((e = launch_reduce(cfg, Epart, n_tiles_h(c), gpart, n_tiles_a(c),
                           static_cast<const int32_t *>(dptr(c, "op_tiles")), K,
                           static_cast<const int32_t *>(dptr(c, "k_ptr")),
                           static_cast<const int32_t *>(dptr(c, "k_ops")), d_op_scale, c->shift,
                           c->prec ? 1 : 0, dE, dG)) !=
        cudaSuccess)
        return cuda_fail(c, e, "reduce kernel");
    ++c->launches;
    c->prof.launches[UCCSD_K_REDUCE]++;
    mk.finish();
    c->state_valid = (grad == nullptr);
    c->last_stream = stream;
    if (!on_dev) {
        e = cudaMemcpyAsync(E, dE, sizeof(double) * B, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess && grad)
            e = cudaMemcpyAsync(grad, dG, sizeof(double) * B * K, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "result download");
    }
    return UCCSD_OK;
}

uccsd_status eval(uccsd_ctx *c, int B, const double *theta, int on_dev, double *E, double *grad,
                  void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (!c->have_exc) return fail(c, UCCSD_ERR_STATE, "set_excitations must come first");
    if (B < 1 || B > c->B) return fail(c, UCCSD_ERR_ARG, "batch size outside the reserved slots");
    if ((!theta && c->K > 0) || !E) return fail(c, UCCSD_ERR_ARG, "null theta or E");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c->prec) return run_eval<float>(c, B, theta, on_dev, E, grad, s);
    return run_eval<double>(c, B, theta, on_dev, E, grad, s);
}

// Precomputed pair lists of a plan (sweeps over lists instead of building
// side lists per factor): at most kMaxListPairs pairs (8 bytes each) per
// plan, larger plans keep the builder kernels.  Lists depend only on the
// plan, so a process-wide cache keyed by a hash of the plan serves repeated
// contexts of the same shape.
constexpr size_t kMaxListPairs = size_t(16) << 20;

uint64_t plan_hash(const uccsd_ctx *c, const SweepPlan &pl) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    const int hdr[4] = {c->n, c->n_alpha, c->n_beta, c->prec};
    mix(hdr, sizeof(hdr));
    for (CRunDev r : pl.runs) {
        r.pl_base = 0;
        mix(&r, sizeof(r));
    }
    mix(pl.ops.data(), pl.ops.size() * sizeof(COpDev));
    return h;
}

// One device copy of a plan's pair lists, shared by every context on that
// device whose plan has the same hash.  Freed when the cache has dropped the
// plan and no context holds it.
struct DeviceLists {
    int device = -1;
    void *op_pl = nullptr, *pairs = nullptr;
    size_t bytes = 0;
    ~DeviceLists() {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) return;
        cudaSetDevice(device);
        if (op_pl) cudaFree(op_pl);
        if (pairs) cudaFree(pairs);
        cudaSetDevice(cur);
        cudaGetLastError();
    }
};

struct ListEntry {
    std::shared_ptr<PairLists> lists;  // null: over the size limit
    std::vector<int32_t> pl_base;
    std::mutex dev_mu;
    std::vector<std::shared_ptr<DeviceLists>> dev;  // by device, uploaded on first use
};

std::mutex g_list_mu;
// most recent last, at most 32; never destroyed (no CUDA calls at exit)
auto *g_list_cache = new std::vector<std::pair<uint64_t, std::shared_ptr<ListEntry>>>();

std::shared_ptr<ListEntry> cached_lists(const uccsd_ctx *c, SweepPlan *pl, uint64_t key) {
    {
        std::lock_guard<std::mutex> lk(g_list_mu);
        for (auto &kv : *g_list_cache)
            if (kv.first == key) return kv.second;
    }
    auto ent = std::make_shared<ListEntry>();
    auto L = std::make_shared<PairLists>();
    // 8-byte amplitudes: 16 lanes per shared-memory wavefront; 16-byte: 8
    if (build_pair_lists(c->n, c->n_alpha, c->n_beta, kMaxListPairs, pl, L.get(), c->prec ? 16 : 8))
        ent->lists = L;
    for (const CRunDev &r : pl->runs) ent->pl_base.push_back(r.pl_base);
    std::lock_guard<std::mutex> lk(g_list_mu);
    for (auto &kv : *g_list_cache)
        if (kv.first == key) return kv.second;  // another thread built it meanwhile
    g_list_cache->emplace_back(key, ent);
    if (g_list_cache->size() > 32) g_list_cache->erase(g_list_cache->begin());
    return ent;
}

// The device copy of an entry's lists on c's device, uploaded once (a
// synchronous copy: no context may see the lists before they are complete).
uccsd_status device_lists(uccsd_ctx *c, ListEntry &ent, std::shared_ptr<DeviceLists> *out) {
    std::lock_guard<std::mutex> lk(ent.dev_mu);
    if (ent.dev.size() <= size_t(c->device)) ent.dev.resize(c->device + 1);
    if (!ent.dev[c->device]) {
        const PairLists &L = *ent.lists;
        auto d = std::make_shared<DeviceLists>();
        d->device = c->device;
        const size_t b1 = sizeof(int32_t) * std::max<size_t>(L.op_pl.size(), 1);
        // 16 bytes of padding: L2 prefetches round list ranges out to 16-byte boundaries
        const size_t b2 = sizeof(uint32_t) * std::max<size_t>(L.pairs.size(), 1) + 16;
        cudaError_t e = cudaMalloc(&d->op_pl, b1);
        if (e == cudaSuccess) e = cudaMalloc(&d->pairs, b2);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, UCCSD_ERR_OOM, "cudaMalloc of the shared pair lists failed");
        }
        d->bytes = b1 + b2;
        if (!L.op_pl.empty())
            e = cudaMemcpy(d->op_pl, L.op_pl.data(), sizeof(int32_t) * L.op_pl.size(),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !L.pairs.empty())
            e = cudaMemcpy(d->pairs, L.pairs.data(), sizeof(uint32_t) * L.pairs.size(),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "pair-list upload");
        ent.dev[c->device] = d;
    }
    *out = ent.dev[c->device];
    return UCCSD_OK;
}

// Attach pair lists to a plan and its sweep arguments (slot 0 forward,
// 1 adjoint).  Without lists (too large, or beyond the context's HBM budget)
// the plan keeps the builder kernels.
uccsd_status attach_lists(uccsd_ctx *c, SweepPlan *pl, SweepArgs *args, int slot) {
    args->op_pl = nullptr;
    args->pairs = nullptr;
    const uint64_t key = plan_hash(c, *pl);
    std::shared_ptr<ListEntry> ent = cached_lists(c, pl, key);
    auto no_lists = [&] {
        for (CRunDev &r : pl->runs) r.pl_base = -1;
        c->lists_held[slot].reset();
        c->list_key[slot] = 0;
        return UCCSD_OK;
    };
    if (!ent->lists) return no_lists();
    std::shared_ptr<DeviceLists> d;
    if (c->list_key[slot] == key && c->lists_held[slot]) {
        d = std::static_pointer_cast<DeviceLists>(c->lists_held[slot]);
    } else {
        uccsd_status st = device_lists(c, *ent, &d);
        if (st) return st;
        if (c->budget && c->bytes + d->bytes > c->budget) return no_lists();
        c->lists_held[slot] = d;
        c->list_key[slot] = key;
    }
    for (size_t r = 0; r < pl->runs.size(); ++r) pl->runs[r].pl_base = ent->pl_base[r];
    args->op_pl = static_cast<const int2 *>(d->op_pl);
    args->pairs = static_cast<const uint2 *>(d->pairs);
    return UCCSD_OK;
}

// Plan of the Trotter-free ansatz: every excitation once, two vectors (u
// read, w accumulated) per shared-memory tile.
uccsd_status prepare_trotter_free(uccsd_ctx *c) {
    if (c->tf_ready) return UCCSD_OK;
    const int n = c->n;
    const size_t A = amp_bytes(c);
    std::vector<int32_t> ident(c->K);
    for (int k = 0; k < c->K; ++k) ident[k] = k;
    c->tf = plan_sweep(n, c->n_alpha, c->n_beta, A, 2, kSweepBudget, c->exc, ident);
    for (const CRunDev &r : c->tf.runs)
        if ((size_t)r.max_entries * A * 2 > kSweepBudget)
            return fail(c, UCCSD_ERR_ARG, "an excitation does not fit one shared-memory tile");
    uccsd_status st;
    COpDev *p1;
    uint32_t *p4;
    void *p;
    if ((st = upload(c, "tf_ops", c->tf.ops, &p1))) return st;
    if ((st = upload(c, "tf_spread", c->tf.spread, &p4))) return st;
    c->tf_args = c->fwd_args;
    c->tf_args.spread = p4;
    c->tf_args.op_pl = nullptr;
    c->tf_args.pairs = nullptr;
    if ((st = dalloc(c, "tf_coef", sizeof(double) * std::max(c->K, 1), &p))) return st;
    for (const char *name : {"tf_u", "tf_w"}) {
        if ((st = dalloc(c, name, state_elems(c) * amp_bytes(c), &p))) return st;
        // only electron-sector entries are ever written; the rest stays zero
        cudaError_t e = cudaMemsetAsync(p, 0, state_elems(c) * amp_bytes(c), c->setup);
        if (e == cudaSuccess) e = setup_sync(c);
        if (e != cudaSuccess) return cuda_fail(c, e, "memset");
    }
    if ((st = dalloc(c, "tf_grad", sizeof(double) * std::max(c->K, 1), &p))) return st;
    if ((st = dalloc(c, "tf_gpart", sizeof(double) * std::max(c->K, 1) * c->tf.max_tiles, &p)))
        return st;
    int32_t *p2;
    if ((st = upload(c, "tf_op_tiles", c->tf.op_tiles, &p2))) return st;
    c->tf_ready = true;
    return UCCSD_OK;
}

// Truncated Taylor series of exp(A) v in s steps of m terms each.  A is real
// antisymmetric with ||A||_2 <= b = sum_k |theta_k| (every G_k has norm 1),
// so the remainder of one step of length h = b/s is at most
// sum_{j>m} h^j/j! <= h^(m+1)/(m+1)! / (1 - h/(m+2)), and each exact step is
// orthogonal, so s steps stay within s times that.  Steps are limited to
// h <= 1 so that the partial sums never exceed e^h times the vector's norm
// (rounding).  Returns the (s, m) of fewest products s*m within tol.
void taylor_schedule(double b, double tol, int *s_out, int *m_out) {
    *s_out = 1;
    *m_out = 0;
    if (!(b > 0.0)) return;
    long long best = -1;
    // log of the bound on s steps; decreasing in s for m >= 1
    auto lbound = [&](long long s, int m) {
        const double h = b / double(s);
        return std::log(double(s)) + (m + 1) * std::log(h) - std::lgamma(m + 2.0) -
               std::log1p(-h / (m + 2.0));
    };
    const long long s_lo = std::max<long long>(1, (long long)std::ceil(b));
    for (int m = 1; m <= 60; ++m) {
        long long lo = s_lo, hi = s_lo << 20;
        if (lbound(hi, m) > std::log(tol)) continue;
        while (lo < hi) {  // smallest s in [s_lo, hi] within tol
            const long long mid = lo + (hi - lo) / 2;
            if (lbound(mid, m) <= std::log(tol)) hi = mid;
            else lo = mid + 1;
        }
        const long long s = lo;
        if (best < 0 || s * m < best) {
            best = s * m;
            *s_out = int(s);
            *m_out = m;
        }
    }
}

// Gauss-Legendre rule of q nodes on [0, 1] (Newton iteration on the
// three-term recurrence of the Legendre polynomials).
void gauss_legendre01(int q, std::vector<double> *x, std::vector<double> *w) {
    x->assign(q, 0.0);
    w->assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double z = std::cos(3.14159265358979323846 * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= q; ++j) {
                const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) p0 = 1.0, p1 = z;
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        (*x)[q - 1 - i] = 0.5 * (1.0 + z);
        (*w)[q - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Nodes of the gradient integral: |f^(r)| <= (2b)^r C for the integrand
// f(tau) = <lambda(tau)|G_k|phi(tau)>, so the q-node Gauss-Legendre error on
// [0, 1], (q!)^4 / ((2q + 1) ((2q)!)^3) max|f^(2q)|, is bounded; the
// smallest q whose doubled bound stays within tol is used.
int gauss_nodes(double b, double C, double tol) {
    for (int q = 1; q < 400; ++q) {
        const double lb = std::log(2.0 * std::max(C, 1e-300)) + 4.0 * std::lgamma(q + 1.0) +
                          2.0 * q * std::log(std::max(2.0 * b, 1e-300)) - std::log(2.0 * q + 1.0) -
                          3.0 * std::lgamma(2.0 * q + 1.0);
        if (lb <= std::log(tol)) return q;
    }
    return 400;
}

// acc <- exp(sign * length * A) acc on the sector, A = sum_k coef_k G_k with
// b = sum_k |coef_k|; t0, t1 are scratch vectors.
template <typename R>
uccsd_status taylor_apply(uccsd_ctx *c, const LaunchCfg &cfg, void *acc, void *t0, void *t1,
                          const double *coef, double sign, double length, double b) {
    int s = 1, m = 0;
    taylor_schedule(b * length, sizeof(R) == 4 ? 0x1p-24 : 0x1p-53, &s, &m);
    if (m == 0) return UCCSD_OK;
    cudaError_t e;
    if ((e = launch_sector_copy<R>(cfg, t0, acc, c->hsec)) != cudaSuccess)
        return cuda_fail(c, e, "sector copy kernel");
    ++c->launches;
    void *bufs[2] = {t0, t1};
    const COpDev *ops = static_cast<const COpDev *>(dptr(c, "tf_ops"));
    // bufs[cur] holds the current term; the last term of a step is replaced
    // by the step's result, which is the first term of the next step
    int cur = 0;
    for (int step = 0; step < s; ++step) {
        for (int j = 1; j <= m; ++j) {
            // u_j = sign * length * A u_{j-1} / (s j); acc += u_j
            const double scale = sign * length / (double(s) * j);
            for (size_t r = 0; r < c->tf.runs.size(); ++r) {
                if ((e = launch_gen_apply<R>(cfg, bufs[cur], bufs[cur ^ 1], c->tf.runs[r], ops, coef,
                                             scale, c->tf_args, r == 0 ? 1 : 0)) != cudaSuccess)
                    return cuda_fail(c, e, "generator-sum kernel");
                ++c->launches;
            }
            if ((e = launch_sector_axpy<R>(cfg, acc, bufs[cur ^ 1], j == m ? bufs[cur] : nullptr,
                                           c->hsec)) != cudaSuccess)
                return cuda_fail(c, e, "sector axpy kernel");
            ++c->launches;
            if (j < m) cur ^= 1;
        }
    }
    return UCCSD_OK;
}

// E (and, with grad_host, dE/dtheta) of exp(A)|HF>, A = sum_k theta_k G_k.
// Gradient (Duhamel): dE/dtheta_k = 2 int_0^1 Re <lambda(tau)|G_k|phi(tau)> dtau
// with phi(tau) = exp(tau A)|HF> and lambda(tau) = exp(tau A) exp(-A) (H - s) psi.
template <typename R>
uccsd_status run_trotter_free(uccsd_ctx *c, const double *theta, double *E, double *grad_host,
                              cudaStream_t stream) {
    LaunchCfg cfg;
    cfg.n = c->n;
    cfg.N = state_elems(c);
    cfg.B = 1;
    cfg.n_ops = c->K;
    cfg.stream = stream;
    cudaError_t e;
    uccsd_status st;
    double *coef = static_cast<double *>(dptr(c, "tf_coef"));
    if (c->K > 0) {
        e = cudaMemcpyAsync(coef, theta, sizeof(double) * c->K, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "theta upload");
    }
    double b = 0.0;
    for (int k = 0; k < c->K; ++k) b += std::fabs(theta[k]);
    void *psi = dptr(c, "psi"), *sig = dptr(c, "sig");
    void *t0 = dptr(c, "tf_u"), *t1 = dptr(c, "tf_w");
    if ((e = launch_sector_init<R>(cfg, psi, t0, c->hsec, c->hf_addr)) != cudaSuccess)
        return cuda_fail(c, e, "sector init kernel");
    ++c->launches;
    if ((st = taylor_apply<R>(c, cfg, psi, t0, t1, coef, 1.0, 1.0, b))) return st;
    const DevHam<R> &H = *reinterpret_cast<const DevHam<R> *>(sizeof(R) == 4 ? (const void *)&c->hf32
                                                                             : (const void *)&c->hf64);
    double *Epart = static_cast<double *>(dptr(c, "Epart"));
    if ((e = launch_happly<R>(cfg, psi, sig, c->LH, H, c->hsec, Epart, grad_host ? 1 : 0)) !=
        cudaSuccess)
        return cuda_fail(c, e, "H-apply kernel");
    ++c->launches;
    double *dE = static_cast<double *>(dptr(c, "E"));
    if ((e = launch_reduce(cfg, Epart, n_tiles_h(c), static_cast<const double *>(dptr(c, "gpart")),
                           n_tiles_a(c), static_cast<const int32_t *>(dptr(c, "op_tiles")), 0,
                           static_cast<const int32_t *>(dptr(c, "k_ptr")),
                           static_cast<const int32_t *>(dptr(c, "k_ops")),
                           static_cast<const double *>(dptr(c, "op_scale")), c->shift,
                           c->prec ? 1 : 0, dE, nullptr)) != cudaSuccess)
        return cuda_fail(c, e, "reduce kernel");
    ++c->launches;
    double *dG = static_cast<double *>(dptr(c, "tf_grad"));
    if (grad_host && c->K > 0) {
        // lambda(0) = exp(-A) sigma, phi(0) = |HF>
        if ((st = taylor_apply<R>(c, cfg, sig, t0, t1, coef, -1.0, 1.0, b))) return st;
        if ((e = launch_sector_init<R>(cfg, psi, t0, c->hsec, c->hf_addr)) != cudaSuccess)
            return cuda_fail(c, e, "sector init kernel");
        ++c->launches;
        double C = std::fabs(c->shift);
        for (const XZTerm &t : c->H.terms) C += std::fabs(t.c);
        const int q = gauss_nodes(b, C, (sizeof(R) == 4 ? 1e-7 : 1e-14) * std::max(1.0, C));
        std::vector<double> xq, wq;
        gauss_legendre01(q, &xq, &wq);
        const COpDev *ops = static_cast<const COpDev *>(dptr(c, "tf_ops"));
        double *gp = static_cast<double *>(dptr(c, "tf_gpart"));
        const int32_t *ot = static_cast<const int32_t *>(dptr(c, "tf_op_tiles"));
        double tau = 0.0;
        for (int i = 0; i < q; ++i) {
            const double dt = xq[i] - tau;
            tau = xq[i];
            if ((st = taylor_apply<R>(c, cfg, psi, t0, t1, coef, 1.0, dt, b))) return st;
            if ((st = taylor_apply<R>(c, cfg, sig, t0, t1, coef, 1.0, dt, b))) return st;
            for (size_t r = 0; r < c->tf.runs.size(); ++r) {
                if ((e = launch_gen_dot<R>(cfg, psi, sig, c->tf.runs[r], ops, c->tf_args, gp,
                                           c->tf.max_tiles)) != cudaSuccess)
                    return cuda_fail(c, e, "gradient-integrand kernel");
                ++c->launches;
            }
            if ((e = launch_tf_grad_accum(cfg, gp, c->tf.max_tiles, ot, c->K, wq[i], dG, i == 0)) !=
                cudaSuccess)
                return cuda_fail(c, e, "gradient accumulation kernel");
            ++c->launches;
        }
    }
    e = cudaMemcpyAsync(E, dE, sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && grad_host && c->K > 0)
        e = cudaMemcpyAsync(grad_host, dG, sizeof(double) * c->K, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "result download");
    c->state_valid = (grad_host == nullptr);
    c->last_stream = stream;
    return UCCSD_OK;
}

uccsd_status trotter_free(uccsd_ctx *c, const double *theta, int on_dev, double *E, double *grad,
                          void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (!c->have_exc) return fail(c, UCCSD_ERR_STATE, "set_excitations must come first");
    if ((!theta && c->K > 0) || !E) return fail(c, UCCSD_ERR_ARG, "null theta or E");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<double> th(c->K);
    if (c->K > 0) {
        if (on_dev) {
            e = cudaMemcpyAsync(th.data(), theta, sizeof(double) * c->K, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(c, e, "theta download");
        } else {
            std::memcpy(th.data(), theta, sizeof(double) * c->K);
        }
    }
    if (!finite_all(th.data(), th.size())) return fail(c, UCCSD_ERR_ARG, "non-finite theta");
    uccsd_status st = prepare_trotter_free(c);
    if (st) return st;
    double Eh = 0.0;
    std::vector<double> gh(grad ? std::max(c->K, 1) : 0);
    double *gp = grad ? gh.data() : nullptr;
    st = c->prec ? run_trotter_free<float>(c, th.data(), &Eh, gp, s)
                 : run_trotter_free<double>(c, th.data(), &Eh, gp, s);
    if (st) return st;
    if (on_dev) {
        e = cudaMemcpyAsync(E, &Eh, sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && grad && c->K > 0)
            e = cudaMemcpyAsync(grad, gh.data(), sizeof(double) * c->K, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "result copy");
    } else {
        *E = Eh;
        if (grad && c->K > 0) std::memcpy(grad, gh.data(), sizeof(double) * c->K);
    }
    return UCCSD_OK;
}
}  // namespace

extern "C" {

uccsd_status uccsd_create(uccsd_ctx **out, int device, uccsd_prec prec, size_t hbm_budget_bytes) {
    if (!out) return UCCSD_ERR_ARG;
    *out = nullptr;
    if (prec != UCCSD_FP64 && prec != UCCSD_FP32_STATE) return UCCSD_ERR_ARG;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) {
        cudaGetLastError();
        return UCCSD_ERR_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return UCCSD_ERR_CUDA;
    {
        // kernel attributes are per device and set once, never while another
        // host thread may be launching the same kernels
        static std::mutex mu;
        static std::vector<char> done;
        std::lock_guard<std::mutex> lk(mu);
        if (done.size() < size_t(nd)) done.resize(nd, 0);
        if (!done[device]) {
            if (configure_kernels() != cudaSuccess) return UCCSD_ERR_CUDA;
            if (configure_sweep_kernels(kSweepBudget) != cudaSuccess) return UCCSD_ERR_CUDA;
            done[device] = 1;
        }
    }
    uccsd_ctx *c = new uccsd_ctx();
    c->device = device;
    c->prec = int(prec);
    c->budget = hbm_budget_bytes;
    if (cudaStreamCreateWithFlags(&c->own_setup, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return UCCSD_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->mark_ev) cudaEventDestroy(c->mark_ev);
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        if (c->aux) cudaStreamDestroy(c->aux);
        if (c->stage_ev) cudaEventDestroy(c->stage_ev);
        cudaStreamDestroy(c->own_setup);
        delete c;
        return UCCSD_ERR_CUDA;
    }
    c->setup = c->own_setup;
    *out = c;
    return UCCSD_OK;
}

void uccsd_destroy(uccsd_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->stage_off > 0) cudaEventSynchronize(c->stage_ev);
    for (auto &kv : c->mem) cudaFree(kv.second.first);
    if (c->stage) cudaFreeHost(c->stage);
    if (c->stage_ev) cudaEventDestroy(c->stage_ev);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->own_setup) cudaStreamDestroy(c->own_setup);
    if (c->gate_ev) {
        // a waiting gate ends by itself (its time limit); wait for it before
        // its status word goes away
        cudaEventSynchronize(c->gate_ev);
        cudaEventDestroy(c->gate_ev);
    }
    uccsd::gate_status_give(c->gate_status);  // back to the process's pool
    opt_rec_give(c->opt_rec);  // the device is idle after the frees above
    delete c;
}

uccsd_status uccsd_set_setup_stream(uccsd_ctx *c, void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "set-up stream switch: cudaSetDevice");
    // staged copies still queued (on the context's own stream) finish first
    if (c->stage_off > 0 && (e = cudaEventSynchronize(c->stage_ev)) != cudaSuccess)
        return cuda_fail(c, e, "set-up stream switch: staging wait");
    if (!c->setup_async && (e = cudaStreamSynchronize(c->setup)) != cudaSuccess)
        return cuda_fail(c, e, "set-up stream switch: stream wait");
    c->stage_off = 0;
    c->setup_async = stream != nullptr;
    c->setup = stream ? static_cast<cudaStream_t>(stream) : c->own_setup;
    return UCCSD_OK;
}

const char *uccsd_last_error(const uccsd_ctx *c) { return c ? c->err.c_str() : "null context"; }

const char *uccsd_status_string(uccsd_status st) {
    switch (st) {
        case UCCSD_OK: return "ok";
        case UCCSD_ERR_ARG: return "invalid argument";
        case UCCSD_ERR_OOM: return "device out of memory";
        case UCCSD_ERR_CUDA: return "CUDA error";
        case UCCSD_ERR_STATE: return "invalid call order or failed context";
        case UCCSD_ERR_TIMEOUT: return "device wait timed out";
        case UCCSD_ERR_BUDGET: return "HBM budget exceeded";
    }
    return "unknown status";
}

uccsd_status uccsd_set_hamiltonian(uccsd_ctx *c, int n_orb, const double *h, const double *eri,
                                   double e_core) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    uccsd_status st = check_hamiltonian_input(c, n_orb, h, eri, e_core);
    if (st) return st;
    CompiledH H;
    std::string err;
    if (!compile_hamiltonian(n_orb, h, eri, e_core, &H, &err)) return fail(c, UCCSD_ERR_ARG, err);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    c->n_orb = n_orb;
    c->n = 2 * n_orb;
    c->H = std::move(H);
    c->LH = 0;
    c->have_h = c->have_ref = c->have_exc = false;
    c->state_valid = false;
    c->shift = 0.0;
    make_fixed_point(c);
    if ((st = upload_tile_tables(c))) return st;
    // only the context's precision is ever used by its kernels
    if (c->prec) {
        if ((st = upload_ham<float>(c, &c->hf32, "h32_"))) return st;
    } else {
        if ((st = upload_ham<double>(c, &c->hf64, "h64_"))) return st;
    }
    c->have_h = true;
    return UCCSD_OK;
}

uccsd_status uccsd_set_layout(uccsd_ctx *c, int layout) {
    if (!c) return UCCSD_ERR_ARG;
    if (layout != UCCSD_LAYOUT_FULL && layout != UCCSD_LAYOUT_SECTOR && layout != UCCSD_LAYOUT_SCBK)
        return fail(c, UCCSD_ERR_ARG,
                    "layout must be UCCSD_LAYOUT_FULL, UCCSD_LAYOUT_SECTOR or UCCSD_LAYOUT_SCBK");
    if (layout == UCCSD_LAYOUT_SCBK && c->have_h && c->n_orb < 2)
        return fail(c, UCCSD_ERR_ARG, "the tapered encoding needs at least 2 orbitals");
    if (c->have_ref) return fail(c, UCCSD_ERR_STATE, "set_layout must come before set_reference");
    c->layout = layout;
    return UCCSD_OK;
}

uccsd_status uccsd_set_reference(uccsd_ctx *c, int n_alpha, int n_beta) {
    if (!c) return UCCSD_ERR_ARG;
    if (!c->have_h) return fail(c, UCCSD_ERR_STATE, "set_hamiltonian must come first");
    if (n_alpha < 0 || n_beta < 0 || n_alpha > c->n_orb || n_beta > c->n_orb)
        return fail(c, UCCSD_ERR_ARG, "electron counts out of range");
    c->n_alpha = n_alpha;
    c->n_beta = n_beta;
    c->hf = uint32_t(hf_bits(n_alpha, n_beta));
    // shift = <HF|H|HF> from the diagonal quadratic form (FP64)
    double sft = c->H.c0;
    for (int q = 0; q < c->n; ++q) {
        if (!((c->hf >> q) & 1u)) continue;
        sft += c->H.diag_a[q];
        for (int r = q + 1; r < c->n; ++r)
            if ((c->hf >> r) & 1u) sft += c->H.diag_b[size_t(q) * c->n + r];
    }
    c->shift = c->H.has_diag ? sft : c->H.c0;
    c->hf32.diag_q0 = shifted_q0(c);
    c->hf64.diag_q0 = shifted_q0(c);
    uccsd_status st = set_row_layout(c);
    if (st) return st;
    c->have_ref = true;
    c->have_exc = false;
    c->state_valid = false;
    return UCCSD_OK;
}

uccsd_status uccsd_build_uccsd_list(int n_orb, int n_alpha, int n_beta, int32_t *out, int cap,
                                    int *n_out) {
    if (n_orb < 1 || n_orb > 15 || n_alpha < 0 || n_beta < 0 || n_alpha > n_orb || n_beta > n_orb ||
        cap < 0 || !n_out || (cap > 0 && !out))
        return UCCSD_ERR_ARG;
    std::vector<int32_t> v = build_uccsd_list(n_orb, n_alpha, n_beta);
    int count = int(v.size() / 4);
    int w = std::min(count, cap);
    if (w > 0) std::memcpy(out, v.data(), sizeof(int32_t) * 4 * w);
    *n_out = count;
    return UCCSD_OK;
}

uccsd_status uccsd_set_excitations(uccsd_ctx *c, int K, const int32_t *ijab, int trotter_order,
                                   int n_slices) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (!c->have_ref) return fail(c, UCCSD_ERR_STATE, "set_reference must come first");
    if (K < 0 || (K > 0 && !ijab)) return fail(c, UCCSD_ERR_ARG, "bad excitation list");
    if (trotter_order != 1 && trotter_order != 2) return fail(c, UCCSD_ERR_ARG, "trotter_order must be 1 or 2");
    if (n_slices < 1 || n_slices > 64) return fail(c, UCCSD_ERR_ARG, "n_slices must be in [1, 64]");
    const int n = c->n;
    if (c->exc_valid && K == c->K && trotter_order == c->order && n_slices == c->M &&
        c->exc_n == n && c->exc_na == c->n_alpha && c->exc_nb == c->n_beta &&
        c->exc_layout == c->layout &&
        (K == 0 || std::memcmp(ijab, c->ijab.data(), sizeof(int32_t) * 4 * size_t(K)) == 0)) {
        // The same reference shape and list as the last call (a refilled
        // context): the plans, schedule tables, pair lists and slots stand.
        // Only the table pointers are refreshed and the state invalidated.
        for (SweepArgs *a : {&c->fwd_args, &c->adj_args}) {
            a->combos = c->comb_combos;
            a->ranks = c->comb_ranks;
            a->comb_offs = c->comb_offs;
            a->aoff = c->hsec.aoff;
            a->boff = c->hsec.boff;
        }
        c->tf_ready = false;
        c->opt_m = 0;
        c->have_exc = true;
        c->state_valid = false;
        return alloc_slots(c);
    }
    c->exc_valid = false;
    std::vector<CompiledExc> exc(K);
    for (int k = 0; k < K; ++k) {
        const int32_t *r = ijab + 4 * k;
        bool single = r[1] < 0;
        auto occ = [&](int q) { return q >= 0 && q < n && ((c->hf >> q) & 1u); };
        auto vir = [&](int q) { return q >= 0 && q < n && !((c->hf >> q) & 1u); };
        bool ok;
        if (single) {
            ok = r[3] < 0 && occ(r[0]) && vir(r[2]) && ((r[0] & 1) == (r[2] & 1));
        } else {
            ok = occ(r[0]) && occ(r[1]) && vir(r[2]) && vir(r[3]) && r[0] != r[1] && r[2] != r[3] &&
                 ((r[0] & 1) + (r[1] & 1) == (r[2] & 1) + (r[3] & 1));
        }
        if (!ok) return fail(c, UCCSD_ERR_ARG, "excitation row " + std::to_string(k) +
                                                   " is not a spin-conserving occupied->virtual excitation");
        std::string err;
        if (!compile_excitation(n, r, &exc[k], &err)) return fail(c, UCCSD_ERR_ARG, err);
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    c->K = K;
    c->order = trotter_order;
    c->M = n_slices;
    c->ijab.assign(ijab, ijab + 4 * size_t(K));
    c->exc = exc;
    c->tf_ready = false;
    c->opt_m = 0;
    build_schedule(K, trotter_order, n_slices, &c->op_k, &c->op_scale);
    const size_t A = c->prec ? 8 : 16;
    c->fwd = plan_sweep(n, c->n_alpha, c->n_beta, A, 1, kSweepBudget, exc, c->op_k);
    // A forward whose whole sector fits one tile would run one CTA per state
    // (64 of 152 SMs at a batch of 64) on a chain of issue-bound factors; at
    // half the tile budget each state spreads over two tiles (two SMs) at the
    // price of a few runs handing the state on (18 qubits: forward 0.44 ->
    // 0.41 ms).  Plans of several runs already have many tiles per run (26
    // qubits: 512) and keep the full budget.
    if (c->fwd.runs.size() == 1 && c->fwd.max_tiles == 1 &&
        size_t(c->hsec.Da) * size_t(c->hsec.Db) >= 4096)
        c->fwd = plan_sweep(n, c->n_alpha, c->n_beta, A, 1, kSweepBudget / 2, exc, c->op_k);
    c->adj = plan_sweep(n, c->n_alpha, c->n_beta, A, 2, kSweepBudget, exc, c->op_k);
    for (const SweepPlan *pl : {&c->fwd, &c->adj})
        for (const CRunDev &r : pl->runs)
            if ((size_t)r.max_entries * A * (pl == &c->adj ? 2 : 1) > kSweepBudget)
                return fail(c, UCCSD_ERR_ARG, "an excitation does not fit one shared-memory tile");
    // per-amplitude CSR of schedule factors (for the gradient sum)
    std::vector<int32_t> k_ptr(K + 1, 0), k_ops;
    for (size_t o = 0; o < c->op_k.size(); ++o) k_ptr[c->op_k[o] + 1]++;
    for (int k = 0; k < K; ++k) k_ptr[k + 1] += k_ptr[k];
    k_ops.resize(c->op_k.size());
    std::vector<int32_t> fill(k_ptr.begin(), k_ptr.end() - 1);
    for (size_t o = 0; o < c->op_k.size(); ++o) k_ops[fill[c->op_k[o]]++] = int32_t(o);
    uccsd_status st;
    COpDev *p1;
    int32_t *p2;
    double *p3;
    uint32_t *p4;
    if ((st = upload(c, "fwd_ops", c->fwd.ops, &p1))) return st;
    if ((st = upload(c, "adj_ops", c->adj.ops, &p1))) return st;
    if ((st = upload(c, "op_k", c->op_k, &p2))) return st;
    if ((st = upload(c, "op_scale", c->op_scale, &p3))) return st;
    if ((st = upload(c, "k_ptr", k_ptr, &p2))) return st;
    if ((st = upload(c, "k_ops", k_ops, &p2))) return st;
    if ((st = upload(c, "op_tiles", c->adj.op_tiles, &p2))) return st;
    // combinatorial rank tables (uploaded with the Hamiltonian)
    SweepArgs base{};
    base.combos = c->comb_combos;
    base.ranks = c->comb_ranks;
    base.comb_offs = c->comb_offs;
    for (int q = 0; q < n; q += 2) base.amask |= 1u << q;
    base.n_alpha = c->n_alpha;
    base.n_beta = c->n_beta;
    base.aoff = c->hsec.aoff;
    base.boff = c->hsec.boff;
    c->fwd_args = base;
    c->adj_args = base;
    if ((st = upload(c, "fwd_spread", c->fwd.spread, &p4))) return st;
    c->fwd_args.spread = p4;
    if ((st = upload(c, "adj_spread", c->adj.spread, &p4))) return st;
    c->adj_args.spread = p4;
    if ((st = attach_lists(c, &c->fwd, &c->fwd_args, 0))) return st;
    if ((st = attach_lists(c, &c->adj, &c->adj_args, 1))) return st;
    if ((st = attach_entry_map(c, &c->fwd, "fwd_emap", &c->fwd_emap))) return st;
    if ((st = attach_entry_map(c, &c->adj, "adj_emap", &c->adj_emap))) return st;
    // gradient partial slots: the pair-list adjoint writes one per (tile, warp)
    {
        const bool lists = c->adj_args.pairs != nullptr;
        int stride = 1;
        for (const CRunDev &r : c->adj.runs) {
            const int per = r.n_tiles * adjoint_partials_per_tile(r, lists);
            stride = std::max(stride, per);
            for (int o = r.op_begin; o < r.op_end; ++o)
                c->adj.op_tiles[c->adj.ops[o].op_s0 & 0x7FFFFFFFu] = per;
        }
        c->adj.max_tiles = stride;
        if ((st = upload(c, "op_tiles", c->adj.op_tiles, &p2))) return st;
    }
    c->have_exc = true;
    c->state_valid = false;
    if ((st = alloc_slots(c))) return st;
    c->exc_valid = true;
    c->exc_n = n;
    c->exc_na = c->n_alpha;
    c->exc_nb = c->n_beta;
    c->exc_layout = c->layout;
    return UCCSD_OK;
}

uccsd_status uccsd_set_batch(uccsd_ctx *c, int B) {
    if (!c) return UCCSD_ERR_ARG;
    if (B < 1 || B > 4096) return fail(c, UCCSD_ERR_ARG, "batch must be in [1, 4096]");
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    int old = c->B;
    c->B = B;
    uccsd_status st = alloc_slots(c);
    if (st) {
        c->B = old;
        alloc_slots(c);
    }
    c->state_valid = false;
    return st;
}

uccsd_status uccsd_energy(uccsd_ctx *c, const double *theta, int on_dev, double *E, void *stream) {
    return eval(c, 1, theta, on_dev, E, nullptr, stream);
}

uccsd_status uccsd_energy_grad(uccsd_ctx *c, const double *theta, int on_dev, double *E, double *grad,
                               void *stream) {
    if (c && c->K > 0 && !grad) return fail(c, UCCSD_ERR_ARG, "null grad");
    double dummy = 0.0;
    return eval(c, 1, theta, on_dev, E, grad ? grad : (on_dev ? nullptr : &dummy), stream);
}

uccsd_status uccsd_energy_grad_batch(uccsd_ctx *c, int B, const double *theta, int on_dev, double *E,
                                     double *grad, void *stream) {
    return eval(c, B, theta, on_dev, E, grad, stream);
}

uccsd_status uccsd_energy_grad_batched(uccsd_ctx *const *ctxs, int B, const double *const *thetas,
                                       double *E, double *const *grads, void *stream) {
    if (B < 0 || (B > 0 && (!ctxs || !thetas || !E))) return UCCSD_ERR_ARG;
    if (B == 0) return UCCSD_OK;
    // every context is checked before anything is enqueued
    for (int i = 0; i < B; ++i) {
        uccsd_ctx *c = ctxs[i];
        if (!c) return UCCSD_ERR_ARG;
        if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
        if (!c->have_exc) return fail(c, UCCSD_ERR_STATE, "set_excitations must come first");
        if (c->K > 0 && !thetas[i]) return fail(c, UCCSD_ERR_ARG, "null theta");
        if (c->device != ctxs[0]->device)
            return fail(c, UCCSD_ERR_ARG, "the contexts of one batched call share a device");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uccsd_ctx *c0 = ctxs[0];
    cudaError_t e = cudaSetDevice(c0->device);
    if (e == cudaSuccess) e = cudaEventRecord(c0->fork_ev, s);
    if (e != cudaSuccess) return cuda_fail(c0, e, "fork event");
    for (int i = 0; i < B; ++i) {
        uccsd_ctx *c = ctxs[i];
        if ((e = cudaStreamWaitEvent(c->aux, c0->fork_ev, 0)) != cudaSuccess)
            return cuda_fail(c, e, "fork wait");
        uccsd_status st = eval(c, 1, thetas[i], 1, E + i, grads ? grads[i] : nullptr, c->aux);
        if (st) return st;
        if ((e = cudaEventRecord(c->join_ev, c->aux)) != cudaSuccess) return cuda_fail(c, e, "join event");
        if ((e = cudaStreamWaitEvent(s, c->join_ev, 0)) != cudaSuccess) return cuda_fail(c, e, "join wait");
    }
    return UCCSD_OK;
}

}  // extern "C"

namespace {
// Capture one B-slot evaluation, followed by one optimiser step when
// opt_step is set, into the context's graph.
uccsd_status capture_graph(uccsd_ctx *c, int B, const double *theta, double *E, double *grad,
                           void *stream, bool opt_step) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->profiling) return fail(c, UCCSD_ERR_STATE, "capture needs profiling off");
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (!c->have_exc) return fail(c, UCCSD_ERR_STATE, "set_excitations must come first");
    if (B < 1 || B > c->B || !E || (!theta && c->K > 0))
        return fail(c, UCCSD_ERR_ARG, "bad capture arguments");
    if (opt_step && c->opt_m == 0) return fail(c, UCCSD_ERR_STATE, "uccsd_opt_init must come first");
    if (opt_step && c->K > 0 && !grad) return fail(c, UCCSD_ERR_ARG, "null grad");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!s) return fail(c, UCCSD_ERR_ARG, "capture needs a non-default stream");
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
    const uint64_t l0 = c->launches;
    uccsd_status st = c->prec ? run_eval<float>(c, B, theta, 1, E, grad, s)
                              : run_eval<double>(c, B, theta, 1, E, grad, s);
    if (st == UCCSD_OK && opt_step) {
        cudaError_t eo = launch_lbfgs(s, c->K, c->opt_m, c->opt_max_step, c->opt_first,
                                      const_cast<double *>(theta), E, grad,
                                      static_cast<double *>(dptr(c, "opt_state")),
                                      opt_meta_ptr(c),
                                      opt_hist_ptr(c), c->opt_steps);
        if (eo != cudaSuccess) st = fail(c, UCCSD_ERR_CUDA, "optimiser kernel in capture");
        else ++c->launches;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    c->graph_kernels = c->launches - l0;  // kernels inside the graph
    c->launches = l0;
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
    c->graph = g;
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    return UCCSD_OK;
}
}  // namespace

extern "C" {

uccsd_status uccsd_capture(uccsd_ctx *c, int B, const double *theta, double *E, double *grad,
                           void *stream) {
    return capture_graph(c, B, theta, E, grad, stream, false);
}

uccsd_status uccsd_capture_vqe_step(uccsd_ctx *c, double *theta, double *E, double *grad,
                                    void *stream) {
    return capture_graph(c, 1, theta, E, grad, stream, true);
}

uccsd_status uccsd_replay(uccsd_ctx *c, void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (!c->graph_exec) return fail(c, UCCSD_ERR_STATE, "no captured graph");
    cudaError_t e = cudaGraphLaunch(c->graph_exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    c->launches += c->graph_kernels;
    c->last_stream = static_cast<cudaStream_t>(stream);
    return UCCSD_OK;
}

uccsd_status uccsd_get_state(uccsd_ctx *c, int slot, double *out, size_t len) {
    if (!c) return UCCSD_ERR_ARG;
    if (!c->have_exc) return fail(c, UCCSD_ERR_STATE, "no state yet");
    if (slot < 0 || slot >= c->B) return fail(c, UCCSD_ERR_ARG, "slot out of range");
    const size_t N = state_elems(c);
    // the 2^n vector, or the 2^(n-2) vector of the tapered encoding
    const size_t Nfull = c->layout == UCCSD_LAYOUT_SCBK ? N : size_t(1) << c->n;
    if (!out || len < 2 * Nfull) return fail(c, UCCSD_ERR_ARG, "output buffer too small");
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
    const char *src = static_cast<const char *>(dptr(c, "psi")) + size_t(slot) * N * amp_bytes(c);
    std::vector<double> dense(c->layout ? 2 * N : 0);
    double *dst = c->layout ? dense.data() : out;
    if (c->prec) {
        std::vector<float> tmp(2 * N);
        e = cudaMemcpyAsync(tmp.data(), src, N * 8, cudaMemcpyDeviceToHost, c->setup);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->setup);
        // real amplitudes held as hi + lo (two FP32 words per slot)
        for (size_t i = 0; i < N; ++i) {
            dst[2 * i] = (double)tmp[2 * i] + (double)tmp[2 * i + 1];
            dst[2 * i + 1] = 0.0;
        }
    } else {
        e = cudaMemcpyAsync(dst, src, N * 16, cudaMemcpyDeviceToHost, c->setup);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->setup);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "state download");
    if (c->layout == UCCSD_LAYOUT_SCBK) {
        // The kernels compute with the Jordan-Wigner signs of the interleaved
        // orbital order (qubit 2p alpha, 2p + 1 beta); the tapered encoding of
        // uccsd_pauli_terms_scbk orders the orbitals up then down.  The two
        // occupation bases differ by the sign of the permutation between the
        // orders: (-1)^(number of occupied pairs beta q < alpha p).
        std::memset(out, 0, sizeof(double) * 2 * Nfull);
        std::vector<uint32_t> ta, tb;
        scbk_addresses(c->n_orb, &ta, &tb);
        for (uint32_t sa = 0; sa < (1u << c->n_orb); ++sa) {
            if (__builtin_popcount(sa) != c->n_alpha) continue;
            for (uint32_t sb = 0; sb < (1u << c->n_orb); ++sb) {
                if (__builtin_popcount(sb) != c->n_beta) continue;
                int inv = 0;
                for (uint32_t w = sb; w; w &= w - 1u)
                    inv += __builtin_popcount(sa >> (__builtin_ctz(w) + 1));
                const double sg = (inv & 1) ? -1.0 : 1.0;
                const size_t x = size_t(ta[sa]) + tb[sb];
                out[2 * x] = sg * dense[2 * x];
                out[2 * x + 1] = sg * dense[2 * x + 1];
            }
        }
    } else if (c->layout == UCCSD_LAYOUT_SECTOR) {
        // scatter the sector array (alpha rank major, strings ascending) to 2^n
        std::memset(out, 0, sizeof(double) * 2 * Nfull);
        std::vector<uint32_t> sa, sb;
        for (uint32_t sv = 0; sv < (1u << c->n_orb); ++sv) {
            if (__builtin_popcount(sv) == c->n_alpha) sa.push_back(sv);
            if (__builtin_popcount(sv) == c->n_beta) sb.push_back(sv);
        }
        auto spread = [](uint32_t sv, int shift) {
            uint32_t x = 0;
            for (int t = 0; sv; ++t, sv >>= 1)
                if (sv & 1u) x |= 1u << (2 * t + shift);
            return x;
        };
        for (size_t ia = 0; ia < sa.size(); ++ia) {
            const uint32_t xa = spread(sa[ia], 0);
            for (size_t ib = 0; ib < sb.size(); ++ib) {
                const size_t x = xa | spread(sb[ib], 1), i = ia * sb.size() + ib;
                out[2 * x] = dense[2 * i];
                out[2 * x + 1] = dense[2 * i + 1];
            }
        }
    }
    return UCCSD_OK;
}

uccsd_status uccsd_info(const uccsd_ctx *c, uccsd_info_t *info) {
    if (!c || !info) return UCCSD_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_qubits = c->n;
    info->n_orb = c->n_orb;
    info->n_alpha = c->n_alpha;
    info->n_beta = c->n_beta;
    info->K = c->K;
    info->n_ops = int(c->op_k.size());
    info->n_groups = int(c->H.groups.size()) + (c->H.has_diag ? 1 : 0);
    info->n_terms = c->H.n_terms;
    info->n_fwd_runs = int(c->fwd.runs.size());
    info->n_adj_runs = int(c->adj.runs.size());
    info->batch = c->B;
    info->precision = c->prec;
    info->layout = c->layout;
    info->device_bytes = c->bytes;
    info->launches = c->launches;
    return UCCSD_OK;
}

uccsd_status uccsd_set_profiling(uccsd_ctx *c, int on) {
    if (!c) return UCCSD_ERR_ARG;
    c->profiling = on != 0;
    std::memset(&c->prof, 0, sizeof(c->prof));
    return UCCSD_OK;
}

uccsd_status uccsd_get_profile(const uccsd_ctx *c, uccsd_profile_t *out) {
    if (!c || !out) return UCCSD_ERR_ARG;
    *out = c->prof;
    return UCCSD_OK;
}

uccsd_status uccsd_mp1_amplitudes(uccsd_ctx *c, double *t, void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (!c->have_exc) return fail(c, UCCSD_ERR_STATE, "set_excitations must come first");
    const int K = c->K;
    if (K == 0) return UCCSD_OK;
    if (!t) return fail(c, UCCSD_ERR_ARG, "null amplitude output");
    // Numerators: at theta = 0 every factor is the identity, so
    // dE/dtheta_k = 2 <HF|H tau_k|HF> (tau_k^dag annihilates |HF>).
    std::vector<double> zero(K, 0.0), g(K, 0.0);
    double E = 0.0;
    uccsd_status st = eval(c, 1, zero.data(), 0, &E, g.data(), stream);
    if (st) return st;
    // Orbital energies (Moller-Plesset partitioning): the Fock diagonal of the
    // reference, read off the diagonal quadratic form of H,
    // eps_P = d_P + sum_{I in HF, I != P} d_{PI}.
    const int n = c->n;
    std::vector<double> eps(n, 0.0);
    if (c->H.has_diag) {
        for (int P = 0; P < n; ++P) {
            double v = c->H.diag_a[P];
            for (int I = 0; I < n; ++I) {
                if (I == P || !((c->hf >> I) & 1u)) continue;
                v += c->H.diag_b[size_t(std::min(P, I)) * n + std::max(P, I)];
            }
            eps[P] = v;
        }
    }
    for (int k = 0; k < K; ++k) {
        const int32_t *r = &c->ijab[4 * size_t(k)];
        double den = eps[r[0]] - eps[r[2]];
        if (r[1] >= 0) den += eps[r[1]] - eps[r[3]];
        if (!(std::fabs(den) > 1e-12))
            return fail(c, UCCSD_ERR_ARG, "excitation row " + std::to_string(k) +
                                              " has a vanishing orbital-energy denominator");
        t[k] = 0.5 * g[k] / den;
    }
    return UCCSD_OK;
}

uccsd_status uccsd_energy_trotter_free(uccsd_ctx *c, const double *theta, int on_dev, double *E,
                                       void *stream) {
    return trotter_free(c, theta, on_dev, E, nullptr, stream);
}

uccsd_status uccsd_energy_grad_trotter_free(uccsd_ctx *c, const double *theta, int on_dev, double *E,
                                            double *grad, void *stream) {
    if (c && c->K > 0 && !grad) return fail(c, UCCSD_ERR_ARG, "null grad");
    return trotter_free(c, theta, on_dev, E, grad, stream);
}

uccsd_status uccsd_opt_init(uccsd_ctx *c, int memory, double max_step, double first_scale,
                            int max_steps) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (!c->have_exc) return fail(c, UCCSD_ERR_STATE, "set_excitations must come first");
    if (memory < 1 || memory > 32 || !(max_step > 0.0) || !(first_scale > 0.0) || max_steps < 1)
        return fail(c, UCCSD_ERR_ARG, "optimiser parameters out of range");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const size_t K = size_t(std::max(c->K, 1));
    void *p;
    uccsd_status st;
    if ((st = dalloc(c, "opt_state", sizeof(double) * (2 * size_t(memory) * K + memory + 3 * K), &p)))
        return st;
    if (!c->opt_rec && max_steps <= kOptRecDoubles - 2) {
        if ((c->opt_rec = opt_rec_take()) &&
            cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->opt_rec_dev), c->opt_rec, 0) != cudaSuccess) {
            cudaGetLastError();
            opt_rec_give(c->opt_rec);
            c->opt_rec = c->opt_rec_dev = nullptr;
        }
    }
    if (c->opt_rec && max_steps > kOptRecDoubles - 2) {  // longer than a record: device buffers
        opt_rec_give(c->opt_rec);
        c->opt_rec = c->opt_rec_dev = nullptr;
    }
    if (c->opt_rec) {
        p = c->opt_rec_dev;
    } else {
        if ((st = dalloc(c, "opt_meta", 4 * sizeof(int), &p))) return st;
        if ((e = cudaMemsetAsync(p, 0, 4 * sizeof(int), c->setup)) != cudaSuccess) return cuda_fail(c, e, "memset");
        if ((st = dalloc(c, "opt_hist", sizeof(double) * max_steps, &p))) return st;
    }
    // zeroed in stream order (a record's meta words and history at once)
    const size_t zb = c->opt_rec ? sizeof(double) * (2 + size_t(max_steps)) : sizeof(double) * max_steps;
    if ((e = cudaMemsetAsync(p, 0, zb, c->setup)) != cudaSuccess) return cuda_fail(c, e, "memset");
    if ((e = setup_sync(c)) != cudaSuccess) return cuda_fail(c, e, "memset");
    c->opt_m = memory;
    c->opt_steps = max_steps;
    c->opt_max_step = max_step;
    c->opt_first = first_scale;
    return UCCSD_OK;
}

uccsd_status uccsd_opt_step(uccsd_ctx *c, double *theta, const double *E, const double *grad,
                            void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) return fail(c, UCCSD_ERR_STATE, "context failed earlier: " + c->err);
    if (c->opt_m == 0) return fail(c, UCCSD_ERR_STATE, "uccsd_opt_init must come first");
    if (c->K > 0 && (!theta || !grad)) return fail(c, UCCSD_ERR_ARG, "null theta or grad");
    if (!E) return fail(c, UCCSD_ERR_ARG, "null E");
    cudaError_t e = launch_lbfgs(static_cast<cudaStream_t>(stream), c->K, c->opt_m, c->opt_max_step,
                                 c->opt_first, theta, E, grad, static_cast<double *>(dptr(c, "opt_state")),
                                 opt_meta_ptr(c),
                                 opt_hist_ptr(c), c->opt_steps);
    if (e != cudaSuccess) return cuda_fail(c, e, "optimiser kernel");
    ++c->launches;
    c->last_stream = static_cast<cudaStream_t>(stream);
    return UCCSD_OK;
}

uccsd_status uccsd_opt_history(uccsd_ctx *c, double *E, int cap, int *n_out) {
    if (!c || !n_out || cap < 0 || (cap > 0 && !E)) return UCCSD_ERR_ARG;
    if (c->opt_m == 0) return fail(c, UCCSD_ERR_STATE, "uccsd_opt_init must come first");
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
    if (e == cudaSuccess && c->opt_rec) {
        // the record in host memory: complete once the stream is done
        const volatile int *m = reinterpret_cast<const volatile int *>(c->opt_rec);
        const int done = m[3];
        const int n = std::min(done, c->opt_steps);
        const volatile double *h = c->opt_rec + 2;
        for (int i = 0; i < std::min(n, cap); ++i) E[i] = h[i];
        *n_out = std::max(n, 0);
        return UCCSD_OK;
    }
    int meta[4] = {0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(meta, dptr(c, "opt_meta"), sizeof(meta), cudaMemcpyDeviceToHost, c->setup);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->setup);
    const int n = std::min(meta[3], c->opt_steps);
    if (e == cudaSuccess && cap > 0 && n > 0)
        e = cudaMemcpyAsync(E, dptr(c, "opt_hist"), sizeof(double) * std::min(n, cap),
                            cudaMemcpyDeviceToHost, c->setup);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->setup);
    if (e != cudaSuccess) return cuda_fail(c, e, "optimiser history download");
    *n_out = n;
    return UCCSD_OK;
}

uccsd_status uccsd_hamiltonian_stats(int n_orb, const double *h, const double *eri, double e_core,
                                     int *n_groups, int *n_terms) {
    uccsd_status st = check_hamiltonian_input(nullptr, n_orb, h, eri, e_core);
    if (st) return st;
    CompiledH H;
    std::string err;
    if (!compile_hamiltonian(n_orb, h, eri, e_core, &H, &err)) return UCCSD_ERR_ARG;
    if (n_groups) *n_groups = int(H.groups.size()) + (H.has_diag ? 1 : 0);
    if (n_terms) *n_terms = H.n_terms;
    return UCCSD_OK;
}

uccsd_status uccsd_happly_mixed_order(int n_orb, int n_beta, int32_t *out, int cap, int *n_out) {
    if (n_orb < 1 || n_orb > 15 || n_beta < 0 || n_beta > n_orb || cap < 0 || !n_out ||
        (cap > 0 && !out))
        return UCCSD_ERR_ARG;
    const std::vector<uint8_t> &ord = mixed_order(n_orb, n_beta);
    const size_t w = std::min(size_t(cap), ord.size());
    for (size_t i = 0; i < w; ++i) out[i] = ord[i];
    *n_out = int(ord.size());
    return UCCSD_OK;
}

uccsd_status uccsd_plan_entry_map(int n_orb, int n_alpha, int n_beta, const int32_t *ijab, int K,
                                  int amp_bytes, int nvec, int32_t *out, int cap, int *n_out) {
    if (n_orb < 1 || n_orb > 15 || n_alpha < 0 || n_beta < 0 || n_alpha > n_orb ||
        n_beta > n_orb || K < 1 || !ijab || (amp_bytes != 8 && amp_bytes != 16) ||
        (nvec != 1 && nvec != 2) || cap < 0 || !n_out || (cap > 0 && !out))
        return UCCSD_ERR_ARG;
    const int n = 2 * n_orb;
    const uint64_t hf = hf_bits(n_alpha, n_beta);
    std::vector<CompiledExc> exc(K);
    for (int k = 0; k < K; ++k) {
        const int32_t *r = ijab + 4 * k;
        std::string err;
        auto occ = [&](int q) { return q >= 0 && q < n && ((hf >> q) & 1u); };
        auto vir = [&](int q) { return q >= 0 && q < n && !((hf >> q) & 1u); };
        const bool ok = r[1] < 0 ? r[3] < 0 && occ(r[0]) && vir(r[2]) && ((r[0] & 1) == (r[2] & 1))
                                 : occ(r[0]) && occ(r[1]) && vir(r[2]) && vir(r[3]) && r[0] != r[1] &&
                                       r[2] != r[3] &&
                                       ((r[0] & 1) + (r[1] & 1) == (r[2] & 1) + (r[3] & 1));
        if (!ok || !compile_excitation(n, r, &exc[k], &err)) return UCCSD_ERR_ARG;
    }
    std::vector<int32_t> op_k;
    std::vector<double> op_scale;
    build_schedule(K, 1, 1, &op_k, &op_scale);
    SweepPlan plan = plan_sweep(n, n_alpha, n_beta, size_t(amp_bytes), nvec, kSweepBudget, exc, op_k);
    size_t total = 0;
    for (const CRunDev &r : plan.runs) total += size_t(r.n_tiles) * size_t(r.max_entries);
    if (total > (size_t(1) << 26)) return UCCSD_ERR_ARG;  // a check hook for small plans
    const std::vector<uint32_t> map = build_entry_map(n, n_alpha, n_beta, &plan);
    size_t rows = 0;
    for (size_t ri = 0; ri < plan.runs.size(); ++ri) {
        const CRunDev &r = plan.runs[ri];
        for (int t = 0; t < r.n_tiles; ++t) {
            const std::vector<uint32_t> dets = tile_entry_dets(n, n_alpha, n_beta, r, t);
            for (size_t e = 0; e < dets.size(); ++e, ++rows) {
                if (rows >= size_t(cap)) continue;
                int32_t *row = out + 5 * rows;
                row[0] = int32_t(ri);
                row[1] = t;
                row[2] = int32_t(e);
                row[3] = int32_t(map[size_t(r.emap_base) + size_t(t) * size_t(r.max_entries) + e]);
                row[4] = int32_t(dets[e]);
            }
        }
    }
    *n_out = int(rows);
    return UCCSD_OK;
}

uccsd_status uccsd_plan_pairs(int n_orb, int n_alpha, int n_beta, const int32_t *ijab, int K,
                              int amp_bytes, int nvec, int32_t *out, int cap, int *n_out) {
    if (n_orb < 1 || n_orb > 15 || n_alpha < 0 || n_beta < 0 || n_alpha > n_orb ||
        n_beta > n_orb || K < 1 || !ijab || (amp_bytes != 8 && amp_bytes != 16) ||
        (nvec != 1 && nvec != 2) || cap < 0 || !n_out || (cap > 0 && !out))
        return UCCSD_ERR_ARG;
    const int n = 2 * n_orb;
    const uint64_t hf = hf_bits(n_alpha, n_beta);
    std::vector<CompiledExc> exc(K);
    for (int k = 0; k < K; ++k) {
        const int32_t *r = ijab + 4 * k;
        auto occ = [&](int q) { return q >= 0 && q < n && ((hf >> q) & 1u); };
        auto vir = [&](int q) { return q >= 0 && q < n && !((hf >> q) & 1u); };
        const bool ok = r[1] < 0 ? r[3] < 0 && occ(r[0]) && vir(r[2]) && ((r[0] & 1) == (r[2] & 1))
                                 : occ(r[0]) && occ(r[1]) && vir(r[2]) && vir(r[3]) && r[0] != r[1] &&
                                       r[2] != r[3] &&
                                       ((r[0] & 1) + (r[1] & 1) == (r[2] & 1) + (r[3] & 1));
        std::string err;
        if (!ok || !compile_excitation(n, r, &exc[k], &err)) return UCCSD_ERR_ARG;
    }
    std::vector<int32_t> op_k;
    std::vector<double> op_scale;
    build_schedule(K, 1, 1, &op_k, &op_scale);
    SweepPlan plan = plan_sweep(n, n_alpha, n_beta, size_t(amp_bytes), nvec, kSweepBudget, exc, op_k);
    PairLists L;
    if (!build_pair_lists(n, n_alpha, n_beta, kMaxListPairs, &plan, &L, amp_bytes == 8 ? 16 : 8))
        return UCCSD_ERR_ARG;
    const std::vector<ExpandedPair> pairs = expand_pair_lists(n, n_alpha, n_beta, plan, L);
    const size_t w = std::min(size_t(cap), pairs.size());
    for (size_t i = 0; i < w; ++i) {
        const ExpandedPair &x = pairs[i];
        int32_t *row = out + 7 * i;
        row[0] = x.factor;
        row[1] = int32_t(x.first);
        row[2] = int32_t(x.second);
        row[3] = x.sign;
        row[4] = x.e;
        row[5] = x.e2;
        row[6] = x.index;
    }
    *n_out = int(pairs.size());
    return UCCSD_OK;
}

uccsd_status uccsd_pauli_terms(int n_orb, const double *h, const double *eri, double e_core,
                               uint32_t *xmask, uint32_t *zmask, double *coef, int cap, int *n_out) {
    if (cap < 0 || !n_out || (cap > 0 && (!xmask || !zmask || !coef))) return UCCSD_ERR_ARG;
    uccsd_status st = check_hamiltonian_input(nullptr, n_orb, h, eri, e_core);
    if (st) return st;
    CompiledH H;
    std::string err;
    if (!compile_hamiltonian(n_orb, h, eri, e_core, &H, &err)) return UCCSD_ERR_ARG;
    int w = std::min(cap, H.n_terms);
    for (int t = 0; t < w; ++t) {
        xmask[t] = H.terms[t].x;
        zmask[t] = H.terms[t].z;
        coef[t] = H.terms[t].c;
    }
    *n_out = H.n_terms;
    return UCCSD_OK;
}

}  // extern "C"
