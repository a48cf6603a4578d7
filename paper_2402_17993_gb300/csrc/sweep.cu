// Excitation sweeps over compact electron-sector tiles (sm_103a).
//
// Forward (Eq. 5 / Eq. 6): each run of consecutive schedule factors acts on
// every tile of its bit set T in shared memory.  A CTA owns one tile (fixed
// values `rest` of the bits outside T); the sector leaves (a, b) alpha/beta
// electrons for the tile bits, and the CTA gathers exactly those C(La,a) x
// C(Lb,b) amplitudes from the full 2^n state in HBM, applies all factors of
// the run as parity-signed 2x2 rotations on pairs (x, x ^ flip), and
// scatters them back.  The adjoint sweep does the same backwards on two
// vectors (phi, lambda) and produces per-factor gradient partials.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "amp.cuh"
#include "kernels.cuh"
#include "pdl.cuh"
#include "plan.hpp"

namespace uccsd {
namespace {

constexpr int kSweepThreadsLarge = 512;  // tiles of >= kLargeTile entries
constexpr int kSweepThreadsSmall = 256;
constexpr int kLargeTile = 4096;

template <typename R>
struct Vec2;
template <>
struct Vec2<float> {
    using T = float2;
};
template <>
struct Vec2<double> {
    using T = double2;
};
template <typename R>
using V2 = typename Vec2<R>::T;

__device__ __forceinline__ uint32_t deposit(uint32_t v, uint32_t mask) {
    uint32_t r = 0;
    while (mask) {
        uint32_t low = mask & (0u - mask);
        if (v & 1u) r |= low;
        v >>= 1;
        mask ^= low;
    }
    return r;
}

// Insert a zero bit at each set bit position of mask, lowest first.
__device__ __forceinline__ uint32_t insert_zeros(uint32_t j, uint32_t mask) {
    for (; mask; mask &= mask - 1u) {
        const uint32_t lowm = (mask & (0u - mask)) - 1u;
        j = ((j & ~lowm) << 1) | (j & lowm);
    }
    return j;
}

__device__ __forceinline__ int comb_count(const int32_t *offs, int m, int k) {
    return (k < 0 || k > m) ? 0 : offs[m * 17 + k + 1] - offs[m * 17 + k];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-CTA view of its compact tile.
struct TileView {
    uint32_t rest;
    uint32_t restA, restB;  // orbital strings of the rest bits
    int a, b;            // electrons left for the tile's alpha / beta bits
    int Da, Db;          // C(La, a), C(Lb, b)
    const uint16_t *ca;  // alpha strings of popcount a
    const uint16_t *cb;  // beta strings of popcount b
    const uint16_t *ra;  // rank of an La-bit string in its popcount class
    const uint16_t *rb;
    const uint32_t *spa; // tile alpha string -> orbital string
    const uint32_t *spb;
    const uint32_t *aoff, *boff;  // state addressing
};

__device__ __forceinline__ bool make_view(const CRunDev &run, const SweepArgs &sa, TileView *v) {
    v->rest = deposit(blockIdx.x, run.rmask);
    v->a = sa.n_alpha - __popc(v->rest & sa.amask);
    v->b = sa.n_beta - __popc(v->rest & ~sa.amask);
    if (v->a < 0 || v->a > run.La || v->b < 0 || v->b > run.Lb) return false;
    v->Da = comb_count(sa.comb_offs, run.La, v->a);
    v->Db = comb_count(sa.comb_offs, run.Lb, v->b);
    v->ca = sa.combos + ((1 << run.La) - 1) + sa.comb_offs[run.La * 17 + v->a];
    v->cb = sa.combos + ((1 << run.Lb) - 1) + sa.comb_offs[run.Lb * 17 + v->b];
    v->ra = sa.ranks + ((1 << run.La) - 1);
    v->rb = sa.ranks + ((1 << run.Lb) - 1);
    v->spa = sa.spread + run.spread_off;
    v->spb = v->spa + (1 << run.La);
    v->aoff = sa.aoff;
    v->boff = sa.boff;
    uint32_t ra = 0, rb = 0;
    for (uint32_t m = v->rest; m; m &= m - 1u) {
        const int q = __ffs(m) - 1;
        if (q & 1) rb |= 1u << (q >> 1);
        else ra |= 1u << (q >> 1);
    }
    v->restA = ra;
    v->restB = rb;
    return true;
}

// Address of tile entry e in a slot addressed by the tables aoff / boff.
__device__ __forceinline__ uint32_t entry_index_at(const TileView &v, int e, const uint32_t *aoff,
                                                   const uint32_t *boff) {
    const int ia = e / v.Db;
    const int ib = e - ia * v.Db;
    return aoff[v.restA | v.spa[v.ca[ia]]] + boff[v.restB | v.spb[v.cb[ib]]];
}

// Address of tile entry e in a slot of the state.
__device__ __forceinline__ uint32_t entry_index(const TileView &v, int e) {
    return entry_index_at(v, e, v.aoff, v.boff);
}

// This CTA's tile entries in a plan's entry map (their sector indices, one
// coalesced load each instead of the rank and spread table chain), or null.
__device__ __forceinline__ const uint32_t *tile_map(const uint32_t *emap, const CRunDev &run) {
    return (emap && run.emap_base >= 0)
               ? emap + (size_t)run.emap_base + (size_t)blockIdx.x * (size_t)run.max_entries
               : nullptr;
}

// Write a forward tile's entries to where the next run (or the caller, after
// the last run) reads the state.
template <typename R, int THREADS>
__device__ __forceinline__ void store_forward_tile(const TileView &v, int D, const V2<R> *tile,
                                                   const SweepOut &out, const CRunDev &run) {
    V2<R> *op = static_cast<V2<R> *>(out.phi) + (size_t)blockIdx.y * out.N;
    if (const uint32_t *em = tile_map(out.emap, run)) {
        for (int e = threadIdx.x; e < D; e += THREADS) op[__ldg(em + e)] = tile[e];
    } else {
        for (int e = threadIdx.x; e < D; e += THREADS) op[entry_index_at(v, e, out.aoff, out.boff)] = tile[e];
    }
}

// Write an adjoint tile's phi and lambda entries to where the next run reads
// them (nothing after the last run).
template <typename R, int THREADS>
__device__ __forceinline__ void store_adjoint_tile(const TileView &v, int D, const V2<R> *tp,
                                                   const V2<R> *tl, const SweepOut &out,
                                                   const CRunDev &run) {
    if (!out.phi) return;
    V2<R> *op = static_cast<V2<R> *>(out.phi) + (size_t)blockIdx.y * out.N;
    V2<R> *ol = static_cast<V2<R> *>(out.lam) + (size_t)blockIdx.y * out.N;
    const uint32_t *em = tile_map(out.emap, run);
    for (int e = threadIdx.x; e < D; e += THREADS) {
        const uint32_t x = em ? __ldg(em + e) : entry_index_at(v, e, out.aoff, out.boff);
        op[x] = tp[e];
        ol[x] = tl[e];
    }
}

// Read the tile's entries of the vectors at st (and sl) into tp (and tl).
template <typename R, int THREADS>
__device__ __forceinline__ void load_tile(const TileView &v, int D, const uint32_t *em,
                                          const V2<R> *st, V2<R> *tp, const V2<R> *sl, V2<R> *tl) {
    if (em) {
        for (int e = threadIdx.x; e < D; e += THREADS) {
            const uint32_t x = __ldg(em + e);
            tp[e] = st[x];
            if (sl) tl[e] = sl[x];
        }
    } else {
        for (int e = threadIdx.x; e < D; e += THREADS) {
            const uint32_t x = entry_index(v, e);
            tp[e] = st[x];
            if (sl) tl[e] = sl[x];
        }
    }
}

// Pairs of factor `op` inside the tile: occupied-side strings have the op's
// occupied bits set and its other flip bits clear; the remaining free bits
// carry (a - noa) alpha and (b - nob) beta electrons.  The pairs are the
// product of an alpha-side list (Va strings) and a beta-side list (Vb).
struct PairSet {
    int Va, Vb;
    const uint16_t *fa, *fb;  // free-bit strings
};

__device__ __forceinline__ PairSet pair_set(const CRunDev &run, const SweepArgs &sa,
                                            const TileView &v, const COpDev &op) {
    PairSet p;
    const int ma = run.La - __popc(op.fa), mb = run.Lb - __popc(op.fb);
    const int ka = v.a - __popc(op.oa), kb = v.b - __popc(op.ob);
    p.Va = comb_count(sa.comb_offs, ma, ka);
    p.Vb = comb_count(sa.comb_offs, mb, kb);
    p.fa = p.Va ? sa.combos + ((1 << ma) - 1) + sa.comb_offs[ma * 17 + ka] : nullptr;
    p.fb = p.Vb ? sa.combos + ((1 << mb) - 1) + sa.comb_offs[mb * 17 + kb] : nullptr;
    return p;
}

// Side lists of one factor in shared memory: for alpha string ja the row
// offsets of the occupied side and of its partner, for beta string jb the
// column offsets; bit 31 of the first word carries the string's Jordan-Wigner
// parity.  Entry (ja, jb) of the pair set is then
//   e = A[ja].x + B[jb].x,  e' = A[ja].y + B[jb].y  (parity bits removed).
__device__ __forceinline__ void build_sides(const PairSet &p, const TileView &v, const COpDev &op,
                                            int2 *A, int2 *B) {
    for (int t = threadIdx.x; t < p.Va + p.Vb; t += blockDim.x) {
        if (t < p.Va) {
            const uint32_t s = insert_zeros(p.fa[t], op.fa) | op.oa;
            const int par = __popc(s & op.pa) & 1;
            A[t] = make_int2((int)(v.ra[s] * v.Db) | (par << 31), (int)(v.ra[s ^ op.fa] * v.Db));
        } else {
            const int u = t - p.Va;
            const uint32_t s = insert_zeros(p.fb[u], op.fb) | op.ob;
            const int par = __popc(s & op.pb) & 1;
            B[u] = make_int2((int)v.rb[s] | (par << 31), (int)v.rb[s ^ op.fb]);
        }
    }
}

// x with its sign bit flipped when bit 31 of neg is set.
__device__ __forceinline__ float flip_sign(float x, uint32_t neg) {
    return __int_as_float(__float_as_int(x) ^ (int)(neg & 0x80000000u));
}
__device__ __forceinline__ double flip_sign(double x, uint32_t neg) {
    return __hiloint2double(__double2hiint(x) ^ (int)(neg & 0x80000000u), __double2loint(x));
}

// Stage the run's factor descriptors and (small tiles) the combinatorial
// table prefixes into shared memory at `base`; returns the table view the
// CTA uses.  Callers synchronise before use.
__device__ __forceinline__ SweepArgs stage_tables(const CRunDev &run, const SweepArgs &sa,
                                                  const COpDev *ops, unsigned char *base,
                                                  COpDev **sops) {
    const int nops = run.op_end - run.op_begin;
    COpDev *so = reinterpret_cast<COpDev *>(base);
    const uint32_t *gsrc = reinterpret_cast<const uint32_t *>(ops + run.op_begin);
    uint32_t *gdst = reinterpret_cast<uint32_t *>(so);
    for (int t = threadIdx.x; t < nops * 8; t += blockDim.x) gdst[t] = gsrc[t];
    *sops = so;
    SweepArgs la = sa;
    const int lmax = max(run.La, run.Lb);
    if (lmax <= kStageLmax) {
        int32_t *offs = reinterpret_cast<int32_t *>(so + nops);
        const int n_offs = (lmax + 1) * 17;
        uint16_t *cmb = reinterpret_cast<uint16_t *>(offs + n_offs);
        const int n_str = (1 << (lmax + 1)) - 1;
        uint16_t *rnk = cmb + n_str;
        for (int t = threadIdx.x; t < n_offs; t += blockDim.x) offs[t] = sa.comb_offs[t];
        for (int t = threadIdx.x; t < n_str; t += blockDim.x) {
            cmb[t] = sa.combos[t];
            rnk[t] = sa.ranks[t];
        }
        la.comb_offs = offs;
        la.combos = cmb;
        la.ranks = rnk;
    }
    return la;
}

// As stage_tables, with the run's cos/sin values (of slot csb, gathered by
// factor) staged right after the factor descriptors and, when cls_pl is
// given, the tile class's pair-list entries (offset, count) after them.
template <typename R>
__device__ __forceinline__ SweepArgs stage_run(const CRunDev &run, const SweepArgs &sa,
                                               const COpDev *ops, const V2<R> *csb,
                                               unsigned char *base, COpDev **sops, V2<R> **scs,
                                               const int2 *cls_pl = nullptr, int2 **spl = nullptr,
                                               bool signed_sin = false, uint32_t rest = 0u) {
    const int nops = run.op_end - run.op_begin;
    COpDev *so = reinterpret_cast<COpDev *>(base);
    const uint32_t *gsrc = reinterpret_cast<const uint32_t *>(ops + run.op_begin);
    uint32_t *gdst = reinterpret_cast<uint32_t *>(so);
    // signed_sin: the sine carries the factor's sign and the tile's rest
    // parity (the list sweeps' rotation constants, one load per factor), and
    // so does bit 31 of the staged op_s0 (word 7 of a descriptor)
    for (int t = threadIdx.x; t < nops * 8; t += blockDim.x) {
        uint32_t w = gsrc[t];
        if (signed_sin && (t & 7) == 7)
            w ^= (uint32_t)(__popc(rest & gsrc[t - 1]) & 1) << 31;  // word 6: par_rest
        gdst[t] = w;
    }
    V2<R> *c = reinterpret_cast<V2<R> *>(so + nops);
    for (int t = threadIdx.x; t < nops; t += blockDim.x) {
        const COpDev &op = ops[run.op_begin + t];
        V2<R> v = csb[op.op_s0 & 0x7FFFFFFFu];
        if (signed_sin)
            v.y = flip_sign(v.y, (op.op_s0 ^ ((uint32_t)(__popc(rest & op.par_rest) & 1) << 31)) &
                                     0x80000000u);
        c[t] = v;
    }
    *sops = so;
    *scs = c;
    int2 *pl = reinterpret_cast<int2 *>(c + nops);
    if (spl) {
        for (int t = threadIdx.x; t < nops; t += blockDim.x) pl[t] = cls_pl[t];
        *spl = pl;
    }
    SweepArgs la = sa;
    const int lmax = max(run.La, run.Lb);
    if (lmax <= kStageLmax) {
        int32_t *offs = reinterpret_cast<int32_t *>(pl + nops);
        const int n_offs = (lmax + 1) * 17;
        uint16_t *cmb = reinterpret_cast<uint16_t *>(offs + n_offs);
        const int n_str = (1 << (lmax + 1)) - 1;
        uint16_t *rnk = cmb + n_str;
        for (int t = threadIdx.x; t < n_offs; t += blockDim.x) offs[t] = sa.comb_offs[t];
        for (int t = threadIdx.x; t < n_str; t += blockDim.x) {
            cmb[t] = sa.combos[t];
            rnk[t] = sa.ranks[t];
        }
        la.comb_offs = offs;
        la.combos = cmb;
        la.ranks = rnk;
    }
    return la;
}

// j -> (ja, jb) = (j / Vb, j % Vb) by a float reciprocal with an exact fix-up
// (j < 2^24).
__device__ __forceinline__ void split_index(int j, int Vb, float inv, int *ja, int *jb) {
    int q = __float2int_rz(((float)j + 0.5f) * inv);
    if (q * Vb > j) --q;
    if ((q + 1) * Vb <= j) ++q;
    *ja = q;
    *jb = j - q * Vb;
}


// Walk over the pair set j = ja * Vb + jb in steps of THREADS: the step in
// (ja, jb) coordinates is (sq, sr) with THREADS = sq * Vb + sr.
struct PairWalk {
    int ja, jb, sq, sr, Vb;
    __device__ __forceinline__ void init(int j0, int threads, int vb) {
        Vb = vb;
        const float inv = 1.0f / (float)vb;
        split_index(j0, vb, inv, &ja, &jb);
        split_index(threads, vb, inv, &sq, &sr);
    }
    __device__ __forceinline__ void next(int *a, int *b) const {
        int na = *a + sq, nb = *b + sr;
        if (nb >= Vb) {
            nb -= Vb;
            ++na;
        }
        *a = na;
        *b = nb;
    }
};

// Offsets of a pair from its side-list entries: the low 31 bits of the sums
// are the tile entries of the occupied side and its partner; bit 31 of the
// first sum is the XOR of the two strings' Jordan-Wigner parities.
__device__ __forceinline__ void pair_offsets(int2 a2, int2 b2, int *e, int *e2, uint32_t *par) {
    const uint32_t sum = (uint32_t)a2.x + (uint32_t)b2.x;
    *e = (int)(sum & 0x7FFFFFFFu);
    *e2 = a2.y + b2.y;
    *par = sum;
}

// Rounding of the rotations and dot products fixed by explicit intrinsics,
// so every instantiation of a kernel gives the same bits.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Rotation of the pair (x occupied side, y partner) by the factor's angle:
// (c x - s y, c y + s x).
//   FP64 state: c = cos, complex amplitudes.
//   FP32 state (real amplitudes as hi + lo, see amp.cuh): the first
//   argument is d = 1 - cos = 2 sin^2(angle / 2), and the rotation is
//   x' = x - (d x + s y), y' = y - (d y - s x).  c never appears, so its
//   FP32 rounding (up to 3e-8 for a small angle, a norm change of each
//   factor's pairs) does not either; the rounding error of the large
//   subtraction goes to lo (TwoSum), lo itself is updated by the same map.
template <typename R>
__device__ __forceinline__ void rotate_pair(R c, R s, V2<R> &x, V2<R> &y) {
    const V2<R> x0 = x, y0 = y;
    x.x = fma_rn(c, x0.x, -mul_rn(s, y0.x));
    x.y = fma_rn(c, x0.y, -mul_rn(s, y0.y));
    y.x = fma_rn(c, y0.x, mul_rn(s, x0.x));
    y.y = fma_rn(c, y0.y, mul_rn(s, x0.y));
}
template <>
__device__ __forceinline__ void rotate_pair<float>(float d, float s, float2 &x, float2 &y) {
    const float2 x0 = x, y0 = y;
    const float tx = fma_rn(d, x0.x, mul_rn(s, y0.x));
    const float ty = fma_rn(d, y0.x, -mul_rn(s, x0.x));
    float ex, ey;
    amp::two_sum(x0.x, -tx, x.x, ex);
    amp::two_sum(y0.x, -ty, y.x, ey);
    x.y = fma_rn(-d, x0.y, fma_rn(-s, y0.y, __fadd_rn(x0.y, ex)));
    y.y = fma_rn(-d, y0.y, fma_rn(s, x0.y, __fadd_rn(y0.y, ey)));
}

// Gradient partials.  A pair contributes Re(conj(l_x) (G phi)_x +
// conj(l_x') (G phi)_x') / s with (G phi)_x = -s phi_x', (G phi)_x' =
// s phi_x (pair_dot); the partials of a thread and of a warp are summed in
// Part<R>:
//   FP64 state: double;
//   FP32 state: a float2 (hi, lo) unevaluated sum.  pair_dot forms the dot
//   of the real values hi + lo with the rounding errors of its two main
//   products (FMA) and of their difference (TwoSum) in lo, and the sums
//   carry their rounding errors in lo as well, so the partial reaches FP64
//   through FP32 instructions only (GB300's FP64 rate is 1/64 of its FP32
//   rate, and these sums run once per pair).
template <typename R>
struct PartOf {
    using T = R;
};
template <>
struct PartOf<float> {
    using T = float2;
};
template <typename R>
using Part = typename PartOf<R>::T;

template <typename R>
__device__ __forceinline__ Part<R> part_zero() {
    return (R)0;
}
template <>
__device__ __forceinline__ float2 part_zero<float>() {
    return make_float2(0.f, 0.f);
}
__device__ __forceinline__ void part_add(double &acc, double d) { acc += d; }
__device__ __forceinline__ void part_add(float2 &acc, float2 d) {
    float s, e;
    amp::two_sum(acc.x, d.x, s, e);
    acc.y = __fadd_rn(acc.y, __fadd_rn(d.y, e));
    acc.x = s;
}
__device__ __forceinline__ double part_flip(double v, uint32_t neg) { return flip_sign(v, neg); }
__device__ __forceinline__ float2 part_flip(float2 v, uint32_t neg) {
    return make_float2(flip_sign(v.x, neg), flip_sign(v.y, neg));
}
__device__ __forceinline__ double part_value(double v) { return v; }
__device__ __forceinline__ double part_value(float2 v) { return amp::value(v); }
__device__ __forceinline__ double part_warp_sum(double v) { return warp_sum(v); }
__device__ __forceinline__ float2 part_warp_sum(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 w;
        w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        part_add(v, w);
    }
    return v;
}

template <typename R>
__device__ __forceinline__ Part<R> pair_dot(V2<R> fx, V2<R> fy, V2<R> lx, V2<R> ly) {
    return fma_rn(ly.x, fx.x, fma_rn(ly.y, fx.y, -fma_rn(lx.x, fy.x, mul_rn(lx.y, fy.y))));
}
template <>
__device__ __forceinline__ float2 pair_dot<float>(float2 fx, float2 fy, float2 lx, float2 ly) {
    // l_x' phi_x - l_x phi_x' of the real values hi + lo
    const float p1 = mul_rn(ly.x, fx.x), e1 = fma_rn(ly.x, fx.x, -p1);
    const float p2 = mul_rn(lx.x, fy.x), e2 = fma_rn(lx.x, fy.x, -p2);
    float h, e;
    amp::two_sum(p1, -p2, h, e);
    const float cross = fma_rn(ly.x, fx.y, fma_rn(ly.y, fx.x, -fma_rn(lx.x, fy.y, mul_rn(lx.y, fy.x))));
    return make_float2(h, __fadd_rn(__fadd_rn(e, __fsub_rn(e1, e2)), cross));
}

// Per-factor header written by the builder warp: pair-set sizes, cos, the
// sin with the factor's sign and the tile's rest-bit parity folded in, and
// (adjoint) the two sign bits separately for the gradient partial.
template <typename R>
struct OpHdr {
    int Va, Vb;
    R ct, st;
    uint32_t opneg, rneg;
};

// The builder warps prepare factor `op` in one buffer: side lists (NB
// builder lanes) and the header (builder lane 0, from its cos/sin value csv).
template <typename R, int NB>
__device__ __forceinline__ void build_factor(const CRunDev &run, const SweepArgs &la,
                                             const TileView &v, const COpDev &op, V2<R> csv,
                                             int2 *lists, OpHdr<R> *hdr, int lane) {
    const PairSet p = pair_set(run, la, v, op);
    int2 *A = lists, *B = lists + p.Va;
    for (int t = lane; t < p.Va + p.Vb; t += NB) {
        if (t < p.Va) {
            const uint32_t s = insert_zeros(p.fa[t], op.fa) | op.oa;
            const int par = __popc(s & op.pa) & 1;
            A[t] = make_int2((int)(v.ra[s] * v.Db) | (par << 31), (int)(v.ra[s ^ op.fa] * v.Db));
        } else {
            const int u = t - p.Va;
            const uint32_t s = insert_zeros(p.fb[u], op.fb) | op.ob;
            const int par = __popc(s & op.pb) & 1;
            B[u] = make_int2((int)v.rb[s] | (par << 31), (int)v.rb[s ^ op.fb]);
        }
    }
    if (lane == 0) {
        OpHdr<R> h;
        h.Va = p.Va;
        h.Vb = p.Vb;
        h.opneg = op.op_s0 & 0x80000000u;
        h.rneg = (uint32_t)(__popc(v.rest & op.par_rest) & 1) << 31;
        h.ct = csv.x;
        h.st = flip_sign(csv.y, h.opneg ^ h.rneg);
        *hdr = h;
    }
}

// Builder warps per CTA of THREADS threads (the last warps of the CTA).
template <int THREADS>
struct Roles {
    static constexpr int kBuildWarps = THREADS >= 512 ? 4 : 2;
    static constexpr int kBuildLanes = 32 * kBuildWarps;
    static constexpr int kCompute = THREADS - kBuildLanes;   // compute threads 0 .. kCompute-1
    static constexpr int kComputeWarps = kCompute / 32;
};

// Forward sweep of one run over one tile.  Warp specialisation: the last
// warps build factor o + 1 (side lists and header) while the other warps
// rotate the pairs of factor o; one barrier per factor separates the two
// buffers.  All cos/sin values of the run are staged in shared memory.
template <typename R, int THREADS>
__global__ void __launch_bounds__(THREADS) forward_sweep_kernel(
    V2<R> *__restrict__ psi, size_t N, CRunDev run, const COpDev *__restrict__ ops,
    const V2<R> *__restrict__ cs, int n_ops, SweepArgs sa, int init_hf, uint32_t hf,
    SweepOut out) {
    pdl_wait();  // the state and the cos/sin values are earlier kernels' output
    using RL = Roles<THREADS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ OpHdr<R> hdr[2];
    V2<R> *tile = reinterpret_cast<V2<R> *>(smem_raw);
    int2 *lists = reinterpret_cast<int2 *>(tile + run.max_entries);  // [2][max_da + max_db]
    const int lstride = run.max_da + run.max_db;
    TileView v;
    if (!make_view(run, sa, &v)) return;  // no sector entries in this tile
    const int b = blockIdx.y;
    COpDev *sops;
    V2<R> *scs;
    const SweepArgs la = stage_run<R>(run, sa, ops, cs + (size_t)b * n_ops,
                                      reinterpret_cast<unsigned char *>(lists + 2 * lstride), &sops, &scs);
    __syncthreads();
    make_view(run, la, &v);
    const bool builder = (int)threadIdx.x >= RL::kCompute;
    const int bl = (int)threadIdx.x - RL::kCompute;  // builder lane
    V2<R> *st = psi + (size_t)b * N;
    const int D = v.Da * v.Db;
    const int nops = run.op_end - run.op_begin;
    if (init_hf) {
        for (int e = threadIdx.x; e < D; e += THREADS)
            tile[e] = V2<R>{(R)(entry_index(v, e) == hf ? 1 : 0), (R)0};
    } else {
        load_tile<R, THREADS>(v, D, tile_map(la.emap, run), st, tile, nullptr, nullptr);
    }
    if (builder && nops > 0)
        build_factor<R, RL::kBuildLanes>(run, la, v, sops[0], scs[0], lists, &hdr[0], bl);
    __syncthreads();
    for (int o = 0; o < nops; ++o) {
        const int buf = o & 1;
        if (builder) {
            if (o + 1 < nops)
                build_factor<R, RL::kBuildLanes>(run, la, v, sops[o + 1], scs[o + 1],
                                                 lists + (buf ^ 1) * lstride, &hdr[buf ^ 1], bl);
        } else {
            const OpHdr<R> h = hdr[buf];
            const int P = h.Va * h.Vb;
            const int2 *A = lists + buf * lstride;
            const int2 *B = A + h.Va;
            if ((int)threadIdx.x < P) {
                PairWalk w;
                w.init(threadIdx.x, RL::kCompute, h.Vb);
                int ja = w.ja, jb = w.jb;
                int j = threadIdx.x;
                // two disjoint pairs per iteration: all loads before any store
                for (; j + RL::kCompute < P; j += 2 * RL::kCompute) {
                    int ja1 = ja, jb1 = jb;
                    w.next(&ja1, &jb1);
                    int e0, f0, e1, f1;
                    uint32_t q0, q1;
                    pair_offsets(A[ja], B[jb], &e0, &f0, &q0);
                    pair_offsets(A[ja1], B[jb1], &e1, &f1, &q1);
                    V2<R> x0 = tile[e0], x1 = tile[f0], u0 = tile[e1], u1 = tile[f1];
                    rotate_pair<R>(h.ct, flip_sign(h.st, q0), x0, x1);
                    rotate_pair<R>(h.ct, flip_sign(h.st, q1), u0, u1);
                    tile[e0] = x0;
                    tile[f0] = x1;
                    tile[e1] = u0;
                    tile[f1] = u1;
                    ja = ja1;
                    jb = jb1;
                    w.next(&ja, &jb);
                }
                if (j < P) {
                    int e0, f0;
                    uint32_t q0;
                    pair_offsets(A[ja], B[jb], &e0, &f0, &q0);
                    V2<R> x0 = tile[e0], x1 = tile[f0];
                    rotate_pair<R>(h.ct, flip_sign(h.st, q0), x0, x1);
                    tile[e0] = x0;
                    tile[f0] = x1;
                }
            }
        }
        __syncthreads();
    }
    store_forward_tile<R, THREADS>(v, D, tile, out, run);
}

// Adjoint sweep of one run over one tile, factors in reverse: the compute
// warps form the gradient partial of factor o and un-rotate phi and lambda
// while the builder warps prepare factor o - 1 and write the partial of
// factor o + 1.
template <typename R, int THREADS>
__global__ void __launch_bounds__(THREADS) adjoint_sweep_kernel(
    V2<R> *__restrict__ phi, V2<R> *__restrict__ lam, size_t N, CRunDev run,
    const COpDev *__restrict__ ops, const V2<R> *__restrict__ cs, int n_ops, SweepArgs sa,
    double *__restrict__ gpart, int tile_stride, SweepOut out) {
    pdl_wait();  // phi, lambda and the partial slots belong to earlier kernels first
    using RL = Roles<THREADS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ OpHdr<R> hdr[2];
    __shared__ double wring[2][32];
    const int b = blockIdx.y;
    TileView v;
    if (!make_view(run, sa, &v)) {
        // all-zero tile: its gradient partials are zero
        for (int o = run.op_begin + threadIdx.x; o < run.op_end; o += THREADS)
            gpart[((size_t)b * n_ops + (ops[o].op_s0 & 0x7FFFFFFFu)) * tile_stride + blockIdx.x] = 0.0;
        return;
    }
    V2<R> *tp = reinterpret_cast<V2<R> *>(smem_raw);
    V2<R> *tl = tp + run.max_entries;
    int2 *lists = reinterpret_cast<int2 *>(tl + run.max_entries);
    const int lstride = run.max_da + run.max_db;
    COpDev *sops;
    V2<R> *scs;
    const SweepArgs la = stage_run<R>(run, sa, ops, cs + (size_t)b * n_ops,
                                      reinterpret_cast<unsigned char *>(lists + 2 * lstride), &sops, &scs);
    __syncthreads();
    make_view(run, la, &v);
    const int D = v.Da * v.Db;
    V2<R> *sp = phi + (size_t)b * N;
    V2<R> *sl = lam + (size_t)b * N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool builder = (int)threadIdx.x >= RL::kCompute;
    const int bl = (int)threadIdx.x - RL::kCompute;  // builder lane
    const int nops = run.op_end - run.op_begin;
    load_tile<R, THREADS>(v, D, tile_map(la.emap, run), sp, tp, sl, tl);
    if (builder && nops > 0)
        build_factor<R, RL::kBuildLanes>(run, la, v, sops[nops - 1], scs[nops - 1], lists, &hdr[0], bl);
    __syncthreads();
    // the first builder warp writes the partial of the previous iteration's
    // factor, summed over the compute warps in a fixed order
    auto flush_partial = [&](int it, int o) {
        double s2 = (lane < RL::kComputeWarps) ? wring[it & 1][lane] : 0.0;
        s2 = warp_sum<double>(s2);
        if (lane == 0)
            gpart[((size_t)b * n_ops + (sops[o].op_s0 & 0x7FFFFFFFu)) * tile_stride + blockIdx.x] = s2;
    };
    int it = 0;
    for (int o = nops - 1; o >= 0; --o, ++it) {
        const int buf = it & 1;
        if (builder) {
            if (it > 0 && bl < 32) flush_partial(it - 1, o + 1);
            if (o - 1 >= 0)
                build_factor<R, RL::kBuildLanes>(run, la, v, sops[o - 1], scs[o - 1],
                                                 lists + (buf ^ 1) * lstride, &hdr[buf ^ 1], bl);
        } else {
            const OpHdr<R> h = hdr[buf];
            const int P = h.Va * h.Vb;
            const int2 *A = lists + buf * lstride;
            const int2 *B = A + h.Va;
            Part<R> part = part_zero<R>();
            if ((int)threadIdx.x < P) {
                PairWalk wk;
                wk.init(threadIdx.x, RL::kCompute, h.Vb);
                int ja = wk.ja, jb = wk.jb;
                int j = threadIdx.x;
                // two disjoint pairs per iteration: all loads before any store;
                // the partial carries the string and rest parities, the
                // factor's own sign is applied to the warp sum
                for (; j + RL::kCompute < P; j += 2 * RL::kCompute) {
                    int ja1 = ja, jb1 = jb;
                    wk.next(&ja1, &jb1);
                    int e0, f0, e1, f1;
                    uint32_t q0, q1;
                    pair_offsets(A[ja], B[jb], &e0, &f0, &q0);
                    pair_offsets(A[ja1], B[jb1], &e1, &f1, &q1);
                    V2<R> fa = tp[e0], fb = tp[f0], la0 = tl[e0], lb0 = tl[f0];
                    V2<R> ga = tp[e1], gb = tp[f1], ma = tl[e1], mb = tl[f1];
                    part_add(part, part_flip(pair_dot<R>(fa, fb, la0, lb0), q0 ^ h.rneg));
                    part_add(part, part_flip(pair_dot<R>(ga, gb, ma, mb), q1 ^ h.rneg));
                    const R s0 = flip_sign(h.st, q0), s1 = flip_sign(h.st, q1);
                    // U(-theta): rotate with -s
                    rotate_pair<R>(h.ct, -s0, fa, fb);
                    rotate_pair<R>(h.ct, -s0, la0, lb0);
                    rotate_pair<R>(h.ct, -s1, ga, gb);
                    rotate_pair<R>(h.ct, -s1, ma, mb);
                    tp[e0] = fa;
                    tp[f0] = fb;
                    tl[e0] = la0;
                    tl[f0] = lb0;
                    tp[e1] = ga;
                    tp[f1] = gb;
                    tl[e1] = ma;
                    tl[f1] = mb;
                    ja = ja1;
                    jb = jb1;
                    wk.next(&ja, &jb);
                }
                if (j < P) {
                    int e0, f0;
                    uint32_t q0;
                    pair_offsets(A[ja], B[jb], &e0, &f0, &q0);
                    V2<R> fa = tp[e0], fb = tp[f0], la0 = tl[e0], lb0 = tl[f0];
                    part_add(part, part_flip(pair_dot<R>(fa, fb, la0, lb0), q0 ^ h.rneg));
                    const R s0 = flip_sign(h.st, q0);
                    rotate_pair<R>(h.ct, -s0, fa, fb);
                    rotate_pair<R>(h.ct, -s0, la0, lb0);
                    tp[e0] = fa;
                    tp[f0] = fb;
                    tl[e0] = la0;
                    tl[f0] = lb0;
                }
            }
            // per-warp partial (FP64, or FP32 hi + lo for the FP32 state),
            // then FP64 across the compute warps
            const Part<R> ws = part_warp_sum(part);
            if (lane == 0) wring[buf][warp] = flip_sign(part_value(ws), h.opneg);
        }
        __syncthreads();
    }
    if (builder && bl < 32 && nops > 0) flush_partial(it - 1, 0);
    store_adjoint_tile<R, THREADS>(v, D, tp, tl, out, run);
}

// ---------------------------------------------------------------------------
// Sweeps over precomputed pair lists (plans whose lists fit the budget).
// Every warp rotates pairs; each thread holds its first pairs of the next
// two factors in registers (loaded two factors ahead), so a factor's
// critical path is the barrier, two shared-memory loads per pair, the
// rotation and the stores.
// ---------------------------------------------------------------------------
// Pairs per thread held in registers, loaded two factors ahead.  Measured on
// 18 qubits, batch 64, FP32, two tiles per state: forward 2 slots 0.379 ms
// against 1: 0.613, 3: 0.447, 4: 0.453, 6: 0.398, 8: 0.410; adjoint 2
// against 3 or 4.
template <typename R>
struct ListPre {
    static constexpr int kFwd = sizeof(R) == 4 ? 2 : 4;
    static constexpr int kAdj = 2;
};

template <int KP>
__device__ __forceinline__ void fetch_pairs(uint2 (&dst)[KP], const uint2 *__restrict__ pairs,
                                            int2 pl, int t, int threads) {
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int j = t + k * threads;
        dst[k] = j < pl.y ? __ldg(pairs + pl.x + j) : make_uint2(0u, 0u);
    }
}

// Bring one factor's pair list into L2 ahead of use: one bulk prefetch
// (cp.async.bulk.prefetch.L2) by one thread, kListAhead factors before the
// list is read, so the register prefetch two factors ahead finds it in L2
// even when the lists were evicted since the last evaluation (they come
// from DRAM otherwise).  The range is widened to 16-byte boundaries, which
// the 16 bytes of padding after the device copy of the lists cover.
constexpr int kListAhead = 6;
__device__ __forceinline__ void prefetch_list_l2(const uint2 *pairs, int2 pl) {
    if (pl.y <= 0) return;
    const uintptr_t a = reinterpret_cast<uintptr_t>(pairs + pl.x) & ~uintptr_t(15);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(pairs + pl.x + pl.y) + 15) & ~uintptr_t(15);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a), "r"((uint32_t)(e - a))
                 : "memory");
}

template <typename R, int THREADS, int KP>
__device__ __forceinline__ void forward_list_step(int o, int nops, V2<R> *tile, const COpDev *sops,
                                                  const V2<R> *scs, const int2 *spl,
                                                  const uint2 *__restrict__ pairs, uint32_t rest,
                                                  uint2 (&cur)[KP], uint2 (&nxt)[KP]) {
    const int t = threadIdx.x;
    if (t == 0 && o + kListAhead < nops) prefetch_list_l2(pairs, spl[o + kListAhead]);
    if (o + 2 < nops) fetch_pairs<KP>(nxt, pairs, spl[o + 2], t, THREADS);
    const int2 pl = spl[o];
    const V2<R> csv = scs[o];  // signed sine (stage_run)
    const R ct = csv.x, st = csv.y;
    (void)sops;
    (void)rest;
    // the prefetched pairs in chunks of two: loads of a chunk before its stores
#pragma unroll
    for (int k0 = 0; k0 < KP; k0 += 2) {
        V2<R> x[2], y[2];
#pragma unroll
        for (int k = k0; k < k0 + 2 && k < KP; ++k)
            if (t + k * THREADS < pl.y) {
                x[k - k0] = tile[cur[k].x];
                y[k - k0] = tile[cur[k].y];
            }
#pragma unroll
        for (int k = k0; k < k0 + 2 && k < KP; ++k)
            if (t + k * THREADS < pl.y) {
                rotate_pair<R>(ct, st, x[k - k0], y[k - k0]);
                tile[cur[k].x] = x[k - k0];
                tile[cur[k].y] = y[k - k0];
            }
    }
    // further pairs: loads issued four at a time
    for (int j0 = t + KP * THREADS; j0 < pl.y; j0 += 4 * THREADS) {
        uint2 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            q[k] = j0 + k * THREADS < pl.y ? __ldg(pairs + pl.x + j0 + k * THREADS) : make_uint2(0u, 0u);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (j0 + k * THREADS < pl.y) {
                V2<R> a = tile[q[k].x], c = tile[q[k].y];
                rotate_pair<R>(ct, st, a, c);
                tile[q[k].x] = a;
                tile[q[k].y] = c;
            }
    }
    __syncthreads();
}

template <typename R, int THREADS>
__global__ void __launch_bounds__(THREADS) forward_list_kernel(
    V2<R> *__restrict__ psi, size_t N, CRunDev run, const COpDev *__restrict__ ops,
    const V2<R> *__restrict__ cs, int n_ops, SweepArgs sa, int init_hf, uint32_t hf,
    SweepOut out) {
    pdl_wait();  // the state and the cos/sin values are earlier kernels' output
    constexpr int KP = ListPre<R>::kFwd;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *tile = reinterpret_cast<V2<R> *>(smem_raw);
    TileView v;
    if (!make_view(run, sa, &v)) return;  // no sector entries in this tile
    const int b = blockIdx.y;
    const int nops = run.op_end - run.op_begin;
    const int cls = v.a * (run.Lb + 1) + v.b;
    COpDev *sops;
    V2<R> *scs;
    int2 *spl;
    const SweepArgs la = stage_run<R>(run, sa, ops, cs + (size_t)b * n_ops,
                                      reinterpret_cast<unsigned char *>(tile + tile_alloc(run.max_entries)),
                                      &sops, &scs, sa.op_pl + run.pl_base + (size_t)cls * nops, &spl,
                                      true, v.rest);
    if (threadIdx.x < kTileScratch)  // padding pairs rotate these zeros
        tile[tile_scratch(run.max_entries) + threadIdx.x] = V2<R>{(R)0, (R)0};
    __syncthreads();
    make_view(run, la, &v);
    V2<R> *st = psi + (size_t)b * N;
    const int D = v.Da * v.Db;
    if (init_hf) {
        for (int e = threadIdx.x; e < D; e += THREADS)
            tile[e] = V2<R>{(R)(entry_index(v, e) == hf ? 1 : 0), (R)0};
    } else {
        load_tile<R, THREADS>(v, D, tile_map(la.emap, run), st, tile, nullptr, nullptr);
    }
    if (threadIdx.x < kListAhead && (int)threadIdx.x < nops) prefetch_list_l2(sa.pairs, spl[threadIdx.x]);
    uint2 p0[KP], p1[KP], p2[KP];
    if (nops > 0) fetch_pairs<KP>(p0, sa.pairs, spl[0], threadIdx.x, THREADS);
    if (nops > 1) fetch_pairs<KP>(p1, sa.pairs, spl[1], threadIdx.x, THREADS);
    __syncthreads();
    for (int o = 0; o < nops; o += 3) {
        forward_list_step<R, THREADS, KP>(o, nops, tile, sops, scs, spl, sa.pairs, v.rest, p0, p2);
        if (o + 1 < nops)
            forward_list_step<R, THREADS, KP>(o + 1, nops, tile, sops, scs, spl, sa.pairs, v.rest, p1, p0);
        if (o + 2 < nops)
            forward_list_step<R, THREADS, KP>(o + 2, nops, tile, sops, scs, spl, sa.pairs, v.rest, p2, p1);
    }
    store_forward_tile<R, THREADS>(v, D, tile, out, run);
}

// A thread's gradient partial of one factor waiting for its warp sum: the
// sum runs during the next factor's step (its shuffles overlap that step's
// shared-memory loads instead of delaying the barrier) and lane 0 writes it
// to the factor's (tile, warp) slot with the tile's rest parity and the
// factor's sign applied.
template <typename R>
struct PendingPart {
    Part<R> part;
    double *dst;  // nullptr: nothing pending
    uint32_t neg;
};
template <typename R>
__device__ __forceinline__ void flush_pending(const PendingPart<R> &p) {
    if (!p.dst) return;  // uniform over the block
    if constexpr (sizeof(R) == 4) {
        // FP32 state: the thread's hi + lo partial as a 64-bit fixed-point
        // integer (unit 2^-40), summed exactly over the warp: integer sums
        // are exact and order-free, and cost 2 shuffles and 2 integer adds
        // per level against 2 shuffles and 8 FP32 operations of a float-float
        // tree.  A partial is a sum of products of normalised amplitudes and
        // components of (H - shift) psi, far inside the +-2^23 range.
        const float2 v = p.part;
        long long q = __float2ll_rn(v.x * 1099511627776.0f) + __float2ll_rn(v.y * 1099511627776.0f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if ((threadIdx.x & 31) == 0) *p.dst = flip_sign((double)q * 9.094947017729282e-13, p.neg);
    } else {
        const Part<R> ws = part_warp_sum(p.part);
        if ((threadIdx.x & 31) == 0) *p.dst = flip_sign(part_value(ws), p.neg);
    }
}

// One adjoint factor over precomputed pairs: un-rotates phi and lambda and
// forms this thread's partial of Re <lambda|G|phi>, left pending in `pend`
// (the previous factor's pending partial is written during this step).
template <typename R, int THREADS, int KP>
__device__ __forceinline__ void adjoint_list_step(int o, int nops, V2<R> *tp, V2<R> *tl,
                                                  const COpDev *sops, const V2<R> *scs,
                                                  const int2 *spl, const uint2 *__restrict__ pairs,
                                                  uint32_t rest, uint2 (&cur)[KP], uint2 (&nxt)[KP],
                                                  double *__restrict__ gp, int tile_stride,
                                                  PendingPart<R> &pend) {
    const int t = threadIdx.x, warp = t >> 5;
    if (t == 0 && o - kListAhead >= 0) prefetch_list_l2(pairs, spl[o - kListAhead]);
    if (o - 2 >= 0) fetch_pairs<KP>(nxt, pairs, spl[o - 2], t, THREADS);
    const int2 pl = spl[o];
    const V2<R> csv = scs[o];  // signed sine (stage_run)
    const R ct = csv.x, st = csv.y;
    Part<R> part = part_zero<R>();
    auto one = [&](uint2 q, V2<R> &fa, V2<R> &fb, V2<R> &la0, V2<R> &lb0) {
        const uint32_t e = q.x, e2 = q.y;
        part_add(part, pair_dot<R>(fa, fb, la0, lb0));
        rotate_pair<R>(ct, -st, fa, fb);
        rotate_pair<R>(ct, -st, la0, lb0);
        tp[e] = fa;
        tp[e2] = fb;
        tl[e] = la0;
        tl[e2] = lb0;
    };
    // the prefetched pairs in chunks of two: loads of a chunk before its
    // stores; the previous factor's warp sum between the first loads and
    // their use
#pragma unroll
    for (int k0 = 0; k0 < KP; k0 += 2) {
        V2<R> f[2], g[2], l[2], m[2];
#pragma unroll
        for (int k = k0; k < k0 + 2 && k < KP; ++k)
            if (t + k * THREADS < pl.y) {
                const uint32_t e = cur[k].x, e2 = cur[k].y;
                f[k - k0] = tp[e];
                g[k - k0] = tp[e2];
                l[k - k0] = tl[e];
                m[k - k0] = tl[e2];
            }
        if (k0 == 0) flush_pending<R>(pend);
        if (t + k0 * THREADS < pl.y) one(cur[k0], f[0], g[0], l[0], m[0]);
        // the second slot behind a warp-uniform branch: warps past the
        // factor's pairs skip it instead of issuing it predicated off
        if (k0 + 1 < KP && (int)(t & ~31) + (k0 + 1) * THREADS < pl.y) {
            if (t + (k0 + 1) * THREADS < pl.y) one(cur[k0 + 1], f[1], g[1], l[1], m[1]);
        }
    }
    // further pairs: loads issued four at a time
    for (int j0 = t + KP * THREADS; j0 < pl.y; j0 += 4 * THREADS) {
        uint2 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            q[k] = j0 + k * THREADS < pl.y ? __ldg(pairs + pl.x + j0 + k * THREADS) : make_uint2(0u, 0u);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (j0 + k * THREADS < pl.y) {
                const uint32_t e = q[k].x, e2 = q[k].y;
                V2<R> fa = tp[e], fb = tp[e2], la0 = tl[e], lb0 = tl[e2];
                one(q[k], fa, fb, la0, lb0);
            }
    }
    // the warp partial (FP64, or FP32 hi + lo for the FP32 state) goes to
    // the factor's (tile, warp) slot; the reduction sums the slots in a
    // fixed order in FP64
    const uint32_t w = sops[o].op_s0;  // sign bit with the rest parity (stage_run)
    pend.part = part;
    pend.dst = gp + (size_t)(w & 0x7FFFFFFFu) * tile_stride + warp;
    pend.neg = w & 0x80000000u;
    (void)rest;
    __syncthreads();
}

template <typename R, int THREADS>
__global__ void __launch_bounds__(THREADS) adjoint_list_kernel(
    V2<R> *__restrict__ phi, V2<R> *__restrict__ lam, size_t N, CRunDev run,
    const COpDev *__restrict__ ops, const V2<R> *__restrict__ cs, int n_ops, SweepArgs sa,
    double *__restrict__ gpart, int tile_stride, SweepOut out) {
    pdl_wait();  // phi, lambda and the partial slots belong to earlier kernels first
    constexpr int KP = ListPre<R>::kAdj;
    constexpr int W = THREADS / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.y;
    TileView v;
    if (!make_view(run, sa, &v)) {
        // all-zero tile: its gradient partials are zero
        for (int i = threadIdx.x; i < (run.op_end - run.op_begin) * W; i += THREADS)
            gpart[((size_t)b * n_ops + (ops[run.op_begin + i / W].op_s0 & 0x7FFFFFFFu)) * tile_stride +
                  (size_t)blockIdx.x * W + i % W] = 0.0;
        return;
    }
    V2<R> *tp = reinterpret_cast<V2<R> *>(smem_raw);
    V2<R> *tl = tp + tile_alloc(run.max_entries);
    const int nops = run.op_end - run.op_begin;
    const int cls = v.a * (run.Lb + 1) + v.b;
    COpDev *sops;
    V2<R> *scs;
    int2 *spl;
    const SweepArgs la = stage_run<R>(run, sa, ops, cs + (size_t)b * n_ops,
                                      reinterpret_cast<unsigned char *>(tl + tile_alloc(run.max_entries)),
                                      &sops, &scs, sa.op_pl + run.pl_base + (size_t)cls * nops, &spl,
                                      true, v.rest);
    if (threadIdx.x < kTileScratch) {  // padding pairs rotate these zeros
        tp[tile_scratch(run.max_entries) + threadIdx.x] = V2<R>{(R)0, (R)0};
        tl[tile_scratch(run.max_entries) + threadIdx.x] = V2<R>{(R)0, (R)0};
    }
    __syncthreads();
    make_view(run, la, &v);
    const int D = v.Da * v.Db;
    V2<R> *sp = phi + (size_t)b * N;
    V2<R> *sl = lam + (size_t)b * N;
    load_tile<R, THREADS>(v, D, tile_map(la.emap, run), sp, tp, sl, tl);
    // gradient partials of this slot and tile: gp[op_index * tile_stride + warp]
    double *gp = gpart + (size_t)b * n_ops * tile_stride + (size_t)blockIdx.x * W;
    if (threadIdx.x < kListAhead && (int)threadIdx.x < nops)
        prefetch_list_l2(sa.pairs, spl[nops - 1 - threadIdx.x]);
    uint2 p0[KP], p1[KP], p2[KP];
    if (nops > 0) fetch_pairs<KP>(p0, sa.pairs, spl[nops - 1], threadIdx.x, THREADS);
    if (nops > 1) fetch_pairs<KP>(p1, sa.pairs, spl[nops - 2], threadIdx.x, THREADS);
    __syncthreads();
    PendingPart<R> pend{part_zero<R>(), nullptr, 0u};
    for (int it = 0; it < nops; it += 3) {
        const int o = nops - 1 - it;
        adjoint_list_step<R, THREADS, KP>(o, nops, tp, tl, sops, scs, spl, sa.pairs, v.rest, p0, p2,
                                          gp, tile_stride, pend);
        if (it + 1 < nops)
            adjoint_list_step<R, THREADS, KP>(o - 1, nops, tp, tl, sops, scs, spl, sa.pairs, v.rest,
                                              p1, p0, gp, tile_stride, pend);
        if (it + 2 < nops)
            adjoint_list_step<R, THREADS, KP>(o - 2, nops, tp, tl, sops, scs, spl, sa.pairs, v.rest,
                                              p2, p1, gp, tile_stride, pend);
    }
    flush_pending<R>(pend);
    store_adjoint_tile<R, THREADS>(v, D, tp, tl, out, run);
}

// Trotter-free ansatz (Eq. 3): w = scale * sum_k coef_k G_k u over the
// factors of one run of a plan that holds every excitation once.  u is read
// only; w is accumulated across the runs of the plan (the first run starts
// from zero).  Per pair (x occupied side, x' partner) with G|x> = s|x'>:
// w_x -= s c u_x', w_x' += s c u_x.
template <typename R, int THREADS>
__global__ void __launch_bounds__(THREADS) gen_apply_kernel(
    const V2<R> *__restrict__ u, V2<R> *__restrict__ w, size_t N, CRunDev run,
    const COpDev *__restrict__ ops, const double *__restrict__ coef, double scale, SweepArgs sa,
    int first_run) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileView v;
    if (!make_view(run, sa, &v)) return;
    V2<R> *tu = reinterpret_cast<V2<R> *>(smem_raw);
    V2<R> *tw = tu + run.max_entries;
    int2 *lists = reinterpret_cast<int2 *>(tw + run.max_entries);
    const int lstride = run.max_da + run.max_db;
    COpDev *sops;
    const SweepArgs la = stage_tables(run, sa, ops, reinterpret_cast<unsigned char *>(lists + 2 * lstride), &sops);
    __syncthreads();
    make_view(run, la, &v);
    const int D = v.Da * v.Db;
    for (int e = threadIdx.x; e < D; e += blockDim.x) {
        const uint32_t x = entry_index(v, e);
        tu[e] = u[x];
        V2<R> z;
        z.x = (R)0;
        z.y = (R)0;
        tw[e] = first_run ? z : w[x];
    }
    const int nops = run.op_end - run.op_begin;
    if (nops > 0) {
        const PairSet p0 = pair_set(run, la, v, sops[0]);
        build_sides(p0, v, sops[0], lists, lists + p0.Va);
    }
    __syncthreads();
    int buf = 0;
    for (int o = 0; o < nops; ++o) {
        const COpDev &op = sops[o];
        const PairSet p = pair_set(run, la, v, op);
        int2 *A = lists + buf * lstride;
        int2 *B = A + p.Va;
        if (o + 1 < nops) {
            const PairSet pn = pair_set(run, la, v, sops[o + 1]);
            int2 *An = lists + (buf ^ 1) * lstride;
            build_sides(pn, v, sops[o + 1], An, An + pn.Va);
        }
        const int P = p.Va * p.Vb;
        if (P > 0) {
            const double c0 = scale * coef[op.op_s0 & 0x7FFFFFFFu];
            const R cc = (R)((op.op_s0 >> 31) ? -c0 : c0);
            const int rpar = __popc(v.rest & op.par_rest) & 1;
            const float inv = 1.0f / (float)p.Vb;
            for (int j = threadIdx.x; j < P; j += blockDim.x) {
                int ja, jb;
                split_index(j, p.Vb, inv, &ja, &jb);
                const int2 a2 = A[ja], b2 = B[jb];
                const int e = (a2.x & 0x7FFFFFFF) + (b2.x & 0x7FFFFFFF);
                const int e2 = a2.y + b2.y;
                const int neg = ((((unsigned)(a2.x ^ b2.x)) >> 31) ^ rpar) & 1;
                const R ss = neg ? -cc : cc;
                const V2<R> u0 = tu[e], u1 = tu[e2];
                V2<R> w0 = tw[e], w1 = tw[e2];
                w0.x -= ss * u1.x;
                w0.y -= ss * u1.y;
                w1.x += ss * u0.x;
                w1.y += ss * u0.y;
                tw[e] = w0;
                tw[e2] = w1;
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    for (int e = threadIdx.x; e < D; e += blockDim.x) w[entry_index(v, e)] = tw[e];
}

// Gradient integrand of the Trotter-free ansatz: per factor of one run and
// per tile, the partial of Re <lambda|G_k|phi> (same pair formula as the
// adjoint sweep, no rotation); tiles without sector entries write zero.
template <typename R, int THREADS>
__global__ void __launch_bounds__(THREADS) gen_dot_kernel(
    const V2<R> *__restrict__ phi, const V2<R> *__restrict__ lam, size_t N, CRunDev run,
    const COpDev *__restrict__ ops, SweepArgs sa, double *__restrict__ gpart, int tile_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double wring[2][32];
    TileView v;
    if (!make_view(run, sa, &v)) {
        for (int o = run.op_begin + threadIdx.x; o < run.op_end; o += blockDim.x)
            gpart[(size_t)(ops[o].op_s0 & 0x7FFFFFFFu) * tile_stride + blockIdx.x] = 0.0;
        return;
    }
    V2<R> *tp = reinterpret_cast<V2<R> *>(smem_raw);
    V2<R> *tl = tp + run.max_entries;
    int2 *lists = reinterpret_cast<int2 *>(tl + run.max_entries);
    const int lstride = run.max_da + run.max_db;
    COpDev *sops;
    const SweepArgs la = stage_tables(run, sa, ops, reinterpret_cast<unsigned char *>(lists + 2 * lstride), &sops);
    __syncthreads();
    make_view(run, la, &v);
    const int D = v.Da * v.Db;
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < D; e += blockDim.x) {
        const uint32_t x = entry_index(v, e);
        tp[e] = phi[x];
        tl[e] = lam[x];
    }
    const int nops = run.op_end - run.op_begin;
    if (nops > 0) {
        const PairSet p0 = pair_set(run, la, v, sops[0]);
        build_sides(p0, v, sops[0], lists, lists + p0.Va);
    }
    __syncthreads();
    int buf = 0;
    for (int o = 0; o < nops; ++o) {
        const COpDev &op = sops[o];
        const PairSet p = pair_set(run, la, v, op);
        int2 *A = lists + buf * lstride;
        int2 *B = A + p.Va;
        if (o + 1 < nops) {
            const PairSet pn = pair_set(run, la, v, sops[o + 1]);
            int2 *An = lists + (buf ^ 1) * lstride;
            build_sides(pn, v, sops[o + 1], An, An + pn.Va);
        }
        const int P = p.Va * p.Vb;
        const int opi = (int)(op.op_s0 & 0x7FFFFFFFu);
        double part = 0.0;
        if (P > 0) {
            const int rpar = __popc(v.rest & op.par_rest) & 1;
            const float inv = 1.0f / (float)p.Vb;
            for (int j = threadIdx.x; j < P; j += blockDim.x) {
                int ja, jb;
                split_index(j, p.Vb, inv, &ja, &jb);
                const int2 a2 = A[ja], b2 = B[jb];
                const int e = (a2.x & 0x7FFFFFFF) + (b2.x & 0x7FFFFFFF);
                const int e2 = a2.y + b2.y;
                const bool neg = ((((unsigned)(a2.x ^ b2.x)) >> 31) ^ rpar) & 1;
                const V2<R> fa = tp[e], fb = tp[e2];
                const V2<R> lx = tl[e], ly = tl[e2];
                // (G phi)_x = -s phi_x', (G phi)_x' = s phi_x
                const double d = amp::re_dot(ly, fa) - amp::re_dot(lx, fb);
                part += neg ? -d : d;
            }
        }
        const double dp = (op.op_s0 >> 31) ? -warp_sum(part) : warp_sum(part);
        const int rb = o & 1;
        if (lane == 0) wring[rb][warp] = dp;
        __syncthreads();
        if (warp == 0) {
            double s2 = (lane < nw) ? wring[rb][lane] : 0.0;
            s2 = warp_sum<double>(s2);
            if (lane == 0) gpart[(size_t)opi * tile_stride + blockIdx.x] = s2;
        }
        buf ^= 1;
    }
}

// g[k] (+)= 2 weight sum_t gpart[k][t] over the op_tiles[k] tiles of factor
// k, one warp per factor in a fixed order (deterministic).
__global__ void tf_grad_accum_kernel(const double *__restrict__ gpart, int tile_stride,
                                     const int32_t *__restrict__ op_tiles, int K, double weight,
                                     double *__restrict__ g, int init) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= K) return;
    double sum = 0.0;
    for (int t = lane; t < op_tiles[k]; t += 32) sum += gpart[(size_t)k * tile_stride + t];
    sum = warp_sum<double>(sum);
    if (lane == 0) g[k] = (init ? 0.0 : g[k]) + 2.0 * weight * sum;
}

// Electron-sector element-wise steps of the Taylor series: x runs over the
// sector entries (alpha string rows x beta string columns).
__device__ __forceinline__ uint32_t sector_index(const HSector &hs, int e) {
    const int ia = e / hs.Db;
    const int ib = e - ia * hs.Db;
    return hs.aoff[hs.astr[ia]] + hs.boff[hs.bstr[ib]];
}

// acc = u = |HF> on the sector.
template <typename R>
__global__ void sector_init_kernel(V2<R> *acc, V2<R> *u, HSector hs, uint32_t hf) {
    const int D = hs.Da * hs.Db;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D; e += gridDim.x * blockDim.x) {
        const uint32_t x = sector_index(hs, e);
        V2<R> val;
        val.x = (R)(x == hf ? 1 : 0);
        val.y = (R)0;
        acc[x] = val;
        u[x] = val;
    }
}

// dst = src on the sector.
template <typename R>
__global__ void sector_copy_kernel(V2<R> *dst, const V2<R> *src, HSector hs) {
    const int D = hs.Da * hs.Db;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D; e += gridDim.x * blockDim.x) {
        const uint32_t x = sector_index(hs, e);
        dst[x] = src[x];
    }
}

// acc += w; if u_out, u_out = acc (the next Taylor step's first term).
template <typename R>
__global__ void sector_axpy_kernel(V2<R> *acc, const V2<R> *w, V2<R> *u_out, HSector hs) {
    const int D = hs.Da * hs.Db;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D; e += gridDim.x * blockDim.x) {
        const uint32_t x = sector_index(hs, e);
        V2<R> a = acc[x];
        const V2<R> d = w[x];
        a.x += d.x;
        a.y += d.y;
        acc[x] = a;
        if (u_out) u_out[x] = a;
    }
}

// |HF> in slot b when the schedule is empty.
template <typename R>
__global__ void set_hf_kernel(V2<R> *psi, size_t N, uint32_t hf) {
    V2<R> one;
    one.x = (R)1;
    one.y = (R)0;
    psi[(size_t)blockIdx.x * N + hf] = one;
}

}  // namespace

template <typename R>
cudaError_t launch_forward_sweep(const LaunchCfg &cfg, void *psi, const CRunDev &run,
                                 const COpDev *ops, const void *cs, const SweepArgs &sa,
                                 int init_hf, uint32_t hf, const SweepOut &out) {
    dim3 grid(run.n_tiles, cfg.B);
    const size_t smem = sweep_smem_bytes(run.max_entries, run.max_da, run.max_db, sizeof(V2<R>), 1,
                                         run.op_end - run.op_begin, max(run.La, run.Lb));
    V2<R> *p = static_cast<V2<R> *>(psi);
    const V2<R> *c = static_cast<const V2<R> *>(cs);
    cudaError_t e = cudaSuccess;
    if (run.pl_base >= 0 && sa.pairs) {
        if (run.max_entries >= kLargeTile)
            e = launch_pdl(forward_list_kernel<R, kSweepThreadsLarge>, grid, dim3(kSweepThreadsLarge), smem, cfg.stream,
                           p, cfg.N, run, ops, c, cfg.n_ops, sa, init_hf, hf, out);
        else
            e = launch_pdl(forward_list_kernel<R, kSweepThreadsSmall>, grid, dim3(kSweepThreadsSmall), smem, cfg.stream,
                           p, cfg.N, run, ops, c, cfg.n_ops, sa, init_hf, hf, out);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    if (run.max_entries >= kLargeTile)
        e = launch_pdl(forward_sweep_kernel<R, kSweepThreadsLarge>, grid, dim3(kSweepThreadsLarge), smem, cfg.stream,
                       p, cfg.N, run, ops, c, cfg.n_ops, sa, init_hf, hf, out);
    else
        e = launch_pdl(forward_sweep_kernel<R, kSweepThreadsSmall>, grid, dim3(kSweepThreadsSmall), smem, cfg.stream,
                       p, cfg.N, run, ops, c, cfg.n_ops, sa, init_hf, hf, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint_sweep(const LaunchCfg &cfg, void *phi, void *lam, const CRunDev &run,
                                 const COpDev *ops, const void *cs, const SweepArgs &sa,
                                 double *gpart, int tile_stride, const SweepOut &out) {
    dim3 grid(run.n_tiles, cfg.B);
    const size_t smem = sweep_smem_bytes(run.max_entries, run.max_da, run.max_db, sizeof(V2<R>), 2,
                                         run.op_end - run.op_begin, max(run.La, run.Lb));
    V2<R> *f = static_cast<V2<R> *>(phi);
    V2<R> *l = static_cast<V2<R> *>(lam);
    const V2<R> *c = static_cast<const V2<R> *>(cs);
    cudaError_t e = cudaSuccess;
    if (run.pl_base >= 0 && sa.pairs) {
        if (run.max_entries >= kLargeTile)
            e = launch_pdl(adjoint_list_kernel<R, kSweepThreadsLarge>, grid, dim3(kSweepThreadsLarge), smem, cfg.stream,
                           f, l, cfg.N, run, ops, c, cfg.n_ops, sa, gpart, tile_stride, out);
        else
            e = launch_pdl(adjoint_list_kernel<R, kSweepThreadsSmall>, grid, dim3(kSweepThreadsSmall), smem, cfg.stream,
                           f, l, cfg.N, run, ops, c, cfg.n_ops, sa, gpart, tile_stride, out);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    if (run.max_entries >= kLargeTile)
        e = launch_pdl(adjoint_sweep_kernel<R, kSweepThreadsLarge>, grid, dim3(kSweepThreadsLarge), smem, cfg.stream,
                       f, l, cfg.N, run, ops, c, cfg.n_ops, sa, gpart, tile_stride, out);
    else
        e = launch_pdl(adjoint_sweep_kernel<R, kSweepThreadsSmall>, grid, dim3(kSweepThreadsSmall), smem, cfg.stream,
                       f, l, cfg.N, run, ops, c, cfg.n_ops, sa, gpart, tile_stride, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename R>
cudaError_t launch_set_hf(const LaunchCfg &cfg, void *psi, uint32_t hf) {
    set_hf_kernel<R><<<cfg.B, 1, 0, cfg.stream>>>(static_cast<V2<R> *>(psi), cfg.N, hf);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gen_apply(const LaunchCfg &cfg, const void *u, void *w, const CRunDev &run,
                             const COpDev *ops, const double *coef, double scale,
                             const SweepArgs &sa, int first_run) {
    dim3 grid(run.n_tiles, 1);
    const size_t smem = sweep_smem_bytes(run.max_entries, run.max_da, run.max_db, sizeof(V2<R>), 2,
                                         run.op_end - run.op_begin, max(run.La, run.Lb));
    const V2<R> *pu = static_cast<const V2<R> *>(u);
    V2<R> *pw = static_cast<V2<R> *>(w);
    if (run.max_entries >= kLargeTile)
        gen_apply_kernel<R, kSweepThreadsLarge><<<grid, kSweepThreadsLarge, smem, cfg.stream>>>(
            pu, pw, cfg.N, run, ops, coef, scale, sa, first_run);
    else
        gen_apply_kernel<R, kSweepThreadsSmall><<<grid, kSweepThreadsSmall, smem, cfg.stream>>>(
            pu, pw, cfg.N, run, ops, coef, scale, sa, first_run);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sector_init(const LaunchCfg &cfg, void *acc, void *u, const HSector &hs,
                               uint32_t hf) {
    const int D = hs.Da * hs.Db;
    const int blocks = std::min((D + 255) / 256, 152 * 8);
    sector_init_kernel<R><<<blocks, 256, 0, cfg.stream>>>(static_cast<V2<R> *>(acc),
                                                          static_cast<V2<R> *>(u), hs, hf);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sector_axpy(const LaunchCfg &cfg, void *acc, const void *w, void *u_out,
                               const HSector &hs) {
    const int D = hs.Da * hs.Db;
    const int blocks = std::min((D + 255) / 256, 152 * 8);
    sector_axpy_kernel<R><<<blocks, 256, 0, cfg.stream>>>(
        static_cast<V2<R> *>(acc), static_cast<const V2<R> *>(w), static_cast<V2<R> *>(u_out), hs);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gen_dot(const LaunchCfg &cfg, const void *phi, const void *lam,
                           const CRunDev &run, const COpDev *ops, const SweepArgs &sa,
                           double *gpart, int tile_stride) {
    dim3 grid(run.n_tiles, 1);
    const size_t smem = sweep_smem_bytes(run.max_entries, run.max_da, run.max_db, sizeof(V2<R>), 2,
                                         run.op_end - run.op_begin, max(run.La, run.Lb));
    const V2<R> *f = static_cast<const V2<R> *>(phi);
    const V2<R> *l = static_cast<const V2<R> *>(lam);
    if (run.max_entries >= kLargeTile)
        gen_dot_kernel<R, kSweepThreadsLarge><<<grid, kSweepThreadsLarge, smem, cfg.stream>>>(
            f, l, cfg.N, run, ops, sa, gpart, tile_stride);
    else
        gen_dot_kernel<R, kSweepThreadsSmall><<<grid, kSweepThreadsSmall, smem, cfg.stream>>>(
            f, l, cfg.N, run, ops, sa, gpart, tile_stride);
    return cudaGetLastError();
}

cudaError_t launch_tf_grad_accum(const LaunchCfg &cfg, const double *gpart, int tile_stride,
                                 const int32_t *op_tiles, int K, double weight, double *g,
                                 int init) {
    if (K <= 0) return cudaSuccess;
    const int warps = 8;
    tf_grad_accum_kernel<<<(K + warps - 1) / warps, warps * 32, 0, cfg.stream>>>(
        gpart, tile_stride, op_tiles, K, weight, g, init);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sector_copy(const LaunchCfg &cfg, void *dst, const void *src, const HSector &hs) {
    const int D = hs.Da * hs.Db;
    const int blocks = std::min((D + 255) / 256, 152 * 8);
    sector_copy_kernel<R><<<blocks, 256, 0, cfg.stream>>>(static_cast<V2<R> *>(dst),
                                                          static_cast<const V2<R> *>(src), hs);
    return cudaGetLastError();
}

int adjoint_partials_per_tile(const CRunDev &run, bool lists) {
    if (!lists || run.pl_base < 0) return 1;
    return (run.max_entries >= kLargeTile ? kSweepThreadsLarge : kSweepThreadsSmall) / 32;
}

cudaError_t configure_sweep_kernels(size_t max_smem) {
    const int bytes = (int)max_smem;
    cudaError_t e = cudaSuccess;
#define UCCSD_SWEEP_ATTR(K)                                                               \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    UCCSD_SWEEP_ATTR((forward_sweep_kernel<float, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((forward_sweep_kernel<float, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((forward_sweep_kernel<double, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((forward_sweep_kernel<double, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((adjoint_sweep_kernel<float, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((adjoint_sweep_kernel<float, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((adjoint_sweep_kernel<double, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((adjoint_sweep_kernel<double, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((forward_list_kernel<float, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((forward_list_kernel<float, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((forward_list_kernel<double, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((forward_list_kernel<double, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((adjoint_list_kernel<float, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((adjoint_list_kernel<float, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((adjoint_list_kernel<double, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((adjoint_list_kernel<double, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((gen_apply_kernel<float, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((gen_apply_kernel<float, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((gen_apply_kernel<double, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((gen_apply_kernel<double, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((gen_dot_kernel<float, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((gen_dot_kernel<float, kSweepThreadsSmall>))
    UCCSD_SWEEP_ATTR((gen_dot_kernel<double, kSweepThreadsLarge>))
    UCCSD_SWEEP_ATTR((gen_dot_kernel<double, kSweepThreadsSmall>))
#undef UCCSD_SWEEP_ATTR
    return e;
}

#define UCCSD_SWEEP_INST(R)                                                                    \
    template cudaError_t launch_forward_sweep<R>(const LaunchCfg &, void *, const CRunDev &,   \
                                                 const COpDev *, const void *,                 \
                                                 const SweepArgs &, int, uint32_t,             \
                                                 const SweepOut &);            \
    template cudaError_t launch_adjoint_sweep<R>(const LaunchCfg &, void *, void *,            \
                                                 const CRunDev &, const COpDev *, const void *, \
                                                 const SweepArgs &, double *, int,             \
                                                 const SweepOut &);                            \
    template cudaError_t launch_set_hf<R>(const LaunchCfg &, void *, uint32_t);                \
    template cudaError_t launch_gen_apply<R>(const LaunchCfg &, const void *, void *,          \
                                             const CRunDev &, const COpDev *, const double *,   \
                                             double, const SweepArgs &, int);                   \
    template cudaError_t launch_sector_init<R>(const LaunchCfg &, void *, void *,              \
                                               const HSector &, uint32_t);                      \
    template cudaError_t launch_sector_axpy<R>(const LaunchCfg &, void *, const void *, void *, \
                                               const HSector &);                                \
    template cudaError_t launch_gen_dot<R>(const LaunchCfg &, const void *, const void *,      \
                                           const CRunDev &, const COpDev *, const SweepArgs &,  \
                                           double *, int);                                      \
    template cudaError_t launch_sector_copy<R>(const LaunchCfg &, void *, const void *,        \
                                               const HSector &);
UCCSD_SWEEP_INST(float)
UCCSD_SWEEP_INST(double)
#undef UCCSD_SWEEP_INST

}  // namespace uccsd
