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

#include <cstdint>

#include "kernels.cuh"

namespace uccsd {
namespace {

constexpr int kSweepThreads = 512;

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

// Insert a zero bit at each ascending position pos[0..nb).
__device__ __forceinline__ uint32_t insert_zeros(uint32_t j, const int32_t *pos, int nb) {
    for (int k = 0; k < nb; ++k) {
        const uint32_t lowm = (1u << pos[k]) - 1u;
        j = ((j & ~lowm) << 1) | (j & lowm);
    }
    return j;
}

__device__ __forceinline__ int comb_count(const int32_t *offs, int m, int k) {
    return (k < 0 || k > m) ? 0 : offs[m * 17 + k + 1] - offs[m * 17 + k];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-CTA view of its compact tile.
struct TileView {
    uint32_t rest;
    int a, b;            // electrons left for the tile's alpha / beta bits
    int Da, Db;          // C(La, a), C(Lb, b)
    const uint16_t *ca;  // alpha strings of popcount a
    const uint16_t *cb;  // beta strings of popcount b
    const uint16_t *ra;  // rank of an La-bit string in its popcount class
    const uint16_t *rb;
    const uint32_t *spa; // alpha string -> global bits
    const uint32_t *spb;
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
    return true;
}

__device__ __forceinline__ uint32_t entry_index(const TileView &v, int e) {
    const int ia = e / v.Db;
    const int ib = e - ia * v.Db;
    return v.rest | v.spa[v.ca[ia]] | v.spb[v.cb[ib]];
}

// Pairs of factor `op` inside the tile: occupied-side strings have the op's
// occupied bits set and its other flip bits clear; the remaining free bits
// carry (a - noa) alpha and (b - nob) beta electrons.
struct PairSet {
    int Va, Vb;
    const uint16_t *fa, *fb;  // free-bit strings
};

__device__ __forceinline__ PairSet pair_set(const CRunDev &run, const SweepArgs &sa,
                                            const TileView &v, const COpDev &op) {
    PairSet p;
    const int ma = run.La - op.nfa, mb = run.Lb - op.nfb;
    const int ka = v.a - op.noa, kb = v.b - op.nob;
    p.Va = comb_count(sa.comb_offs, ma, ka);
    p.Vb = comb_count(sa.comb_offs, mb, kb);
    p.fa = p.Va ? sa.combos + ((1 << ma) - 1) + sa.comb_offs[ma * 17 + ka] : nullptr;
    p.fb = p.Vb ? sa.combos + ((1 << mb) - 1) + sa.comb_offs[mb * 17 + kb] : nullptr;
    return p;
}

// Tile entries (e, e2) of pair j and whether its sign is negated.
__device__ __forceinline__ void pair_entries(const PairSet &p, const TileView &v, const COpDev &op,
                                             const int32_t *posa, const int32_t *posb,
                                             uint32_t rpar, int j, int *e, int *e2, bool *neg) {
    const int ja = j / p.Vb;
    const int jb = j - ja * p.Vb;
    const uint32_t sa = insert_zeros(p.fa[ja], posa, op.nfa) | op.oa;
    const uint32_t sb = insert_zeros(p.fb[jb], posb, op.nfb) | op.ob;
    *e = v.ra[sa] * v.Db + v.rb[sb];
    *e2 = v.ra[sa ^ op.fa] * v.Db + v.rb[sb ^ op.fb];
    *neg = ((__popc(sa & op.pa) + __popc(sb & op.pb) + rpar) & 1u) != 0u;
}

template <typename R>
__global__ void __launch_bounds__(kSweepThreads) forward_sweep_kernel(
    V2<R> *__restrict__ psi, size_t N, CRunDev run, const COpDev *__restrict__ ops,
    const V2<R> *__restrict__ cs, int n_ops, SweepArgs sa, int init_hf, uint32_t hf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *tile = reinterpret_cast<V2<R> *>(smem_raw);
    TileView v;
    if (!make_view(run, sa, &v)) return;  // no sector entries in this tile
    const int b = blockIdx.y;
    V2<R> *st = psi + (size_t)b * N;
    const int D = v.Da * v.Db;
    for (int e = threadIdx.x; e < D; e += blockDim.x) {
        const uint32_t x = entry_index(v, e);
        V2<R> val;
        if (init_hf) {
            val.x = (R)(x == hf ? 1 : 0);
            val.y = (R)0;
        } else {
            val = st[x];
        }
        tile[e] = val;
    }
    __syncthreads();
    for (int o = run.op_begin; o < run.op_end; ++o) {
        const COpDev &op = ops[o];
        const PairSet p = pair_set(run, sa, v, op);
        const int P = p.Va * p.Vb;
        if (P == 0) continue;  // uniform over the CTA
        const V2<R> csv = cs[(size_t)b * n_ops + op.op];
        const R ct = csv.x;
        const R st0 = op.s0 > 0 ? csv.y : -csv.y;
        const uint32_t rpar = __popc(v.rest & op.par_rest) & 1u;
        const int32_t posa[4] = {op.posa[0], op.posa[1], op.posa[2], op.posa[3]};
        const int32_t posb[4] = {op.posb[0], op.posb[1], op.posb[2], op.posb[3]};
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            int e, e2;
            bool neg;
            pair_entries(p, v, op, posa, posb, rpar, j, &e, &e2, &neg);
            const R ss = neg ? -st0 : st0;
            const V2<R> x0 = tile[e], x1 = tile[e2];
            V2<R> y0, y1;
            y0.x = ct * x0.x - ss * x1.x;
            y0.y = ct * x0.y - ss * x1.y;
            y1.x = ct * x1.x + ss * x0.x;
            y1.y = ct * x1.y + ss * x0.y;
            tile[e] = y0;
            tile[e2] = y1;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < D; e += blockDim.x) st[entry_index(v, e)] = tile[e];
}

template <typename R>
__global__ void __launch_bounds__(kSweepThreads) adjoint_sweep_kernel(
    V2<R> *__restrict__ phi, V2<R> *__restrict__ lam, size_t N, CRunDev run,
    const COpDev *__restrict__ ops, const V2<R> *__restrict__ cs, int n_ops, SweepArgs sa,
    double *__restrict__ gpart, int tile_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double wring[2][32];
    const int b = blockIdx.y;
    TileView v;
    if (!make_view(run, sa, &v)) {
        // all-zero tile: its gradient partials are zero
        for (int o = run.op_begin + threadIdx.x; o < run.op_end; o += blockDim.x)
            gpart[((size_t)b * n_ops + ops[o].op) * tile_stride + blockIdx.x] = 0.0;
        return;
    }
    const int D = v.Da * v.Db;
    V2<R> *tp = reinterpret_cast<V2<R> *>(smem_raw);
    V2<R> *tl = tp + run.max_entries;
    V2<R> *sp = phi + (size_t)b * N;
    V2<R> *sl = lam + (size_t)b * N;
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < D; e += blockDim.x) {
        const uint32_t x = entry_index(v, e);
        tp[e] = sp[x];
        tl[e] = sl[x];
    }
    __syncthreads();
    int it = 0;
    for (int o = run.op_end - 1; o >= run.op_begin; --o) {
        const COpDev &op = ops[o];
        const PairSet p = pair_set(run, sa, v, op);
        const int P = p.Va * p.Vb;
        const size_t gidx = ((size_t)b * n_ops + op.op) * tile_stride + blockIdx.x;
        if (P == 0) {
            if (threadIdx.x == 0) gpart[gidx] = 0.0;
            continue;
        }
        const V2<R> csv = cs[(size_t)b * n_ops + op.op];
        const R ct = csv.x;
        const R st0 = op.s0 > 0 ? csv.y : -csv.y;
        const uint32_t rpar = __popc(v.rest & op.par_rest) & 1u;
        const int32_t posa[4] = {op.posa[0], op.posa[1], op.posa[2], op.posa[3]};
        const int32_t posb[4] = {op.posb[0], op.posb[1], op.posb[2], op.posb[3]};
        R part = (R)0;
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            int e, e2;
            bool neg;
            pair_entries(p, v, op, posa, posb, rpar, j, &e, &e2, &neg);
            const V2<R> fa = tp[e], fb = tp[e2];
            const V2<R> la = tl[e], lb = tl[e2];
            // (G phi)_x = -s phi_x', (G phi)_x' = s phi_x
            const R d = (lb.x * fa.x + lb.y * fa.y) - (la.x * fb.x + la.y * fb.y);
            part += neg ? -d : d;
            const R ss = neg ? -st0 : st0;
            V2<R> w;
            w.x = ct * fa.x + ss * fb.x;
            w.y = ct * fa.y + ss * fb.y;
            tp[e] = w;
            w.x = ct * fb.x - ss * fa.x;
            w.y = ct * fb.y - ss * fa.y;
            tp[e2] = w;
            w.x = ct * la.x + ss * lb.x;
            w.y = ct * la.y + ss * lb.y;
            tl[e] = w;
            w.x = ct * lb.x - ss * la.x;
            w.y = ct * lb.y - ss * la.y;
            tl[e2] = w;
        }
        double dp = warp_sum((double)part * (double)op.s0);
        const int buf = it & 1;
        ++it;
        if (lane == 0) wring[buf][warp] = dp;
        __syncthreads();
        if (warp == 0) {
            double s = (lane < nw) ? wring[buf][lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) gpart[gidx] = s;
        }
    }
    for (int e = threadIdx.x; e < D; e += blockDim.x) {
        const uint32_t x = entry_index(v, e);
        sp[x] = tp[e];
        sl[x] = tl[e];
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
                                 int init_hf, uint32_t hf) {
    dim3 grid(run.n_tiles, cfg.B);
    const size_t smem = sizeof(V2<R>) * (size_t)run.max_entries;
    forward_sweep_kernel<R><<<grid, kSweepThreads, smem, cfg.stream>>>(
        static_cast<V2<R> *>(psi), cfg.N, run, ops, static_cast<const V2<R> *>(cs), cfg.n_ops, sa,
        init_hf, hf);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint_sweep(const LaunchCfg &cfg, void *phi, void *lam, const CRunDev &run,
                                 const COpDev *ops, const void *cs, const SweepArgs &sa,
                                 double *gpart, int tile_stride) {
    dim3 grid(run.n_tiles, cfg.B);
    const size_t smem = 2 * sizeof(V2<R>) * (size_t)run.max_entries;
    adjoint_sweep_kernel<R><<<grid, kSweepThreads, smem, cfg.stream>>>(
        static_cast<V2<R> *>(phi), static_cast<V2<R> *>(lam), cfg.N, run, ops,
        static_cast<const V2<R> *>(cs), cfg.n_ops, sa, gpart, tile_stride);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_set_hf(const LaunchCfg &cfg, void *psi, uint32_t hf) {
    set_hf_kernel<R><<<cfg.B, 1, 0, cfg.stream>>>(static_cast<V2<R> *>(psi), cfg.N, hf);
    return cudaGetLastError();
}

cudaError_t configure_sweep_kernels(size_t max_smem) {
    cudaError_t e;
    const int bytes = (int)max_smem;
    if ((e = cudaFuncSetAttribute(forward_sweep_kernel<float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(forward_sweep_kernel<double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(adjoint_sweep_kernel<float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    return cudaFuncSetAttribute(adjoint_sweep_kernel<double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

#define UCCSD_SWEEP_INST(R)                                                                    \
    template cudaError_t launch_forward_sweep<R>(const LaunchCfg &, void *, const CRunDev &,   \
                                                 const COpDev *, const void *,                 \
                                                 const SweepArgs &, int, uint32_t);            \
    template cudaError_t launch_adjoint_sweep<R>(const LaunchCfg &, void *, void *,            \
                                                 const CRunDev &, const COpDev *, const void *, \
                                                 const SweepArgs &, double *, int);            \
    template cudaError_t launch_set_hf<R>(const LaunchCfg &, void *, uint32_t);
UCCSD_SWEEP_INST(float)
UCCSD_SWEEP_INST(double)
#undef UCCSD_SWEEP_INST

}  // namespace uccsd
