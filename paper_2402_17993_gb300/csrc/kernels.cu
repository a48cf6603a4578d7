// UCCSD state-vector kernels for GB300 (sm_103a).
//
// State layout: one slot = 2^n complex amplitudes (float2 or double2),
// slot b at offset b * 2^n; amplitude index x has bit P = occupation of
// spin orbital P.  Nothing here is a dense contraction, so no tensor cores:
// the rotations are bandwidth bound, the Hamiltonian action is ALU bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace uccsd {
namespace {

constexpr int kThreads = 256;

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

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// acc += v * p.  FP32 accumulators carry a Kahan compensation term so that
// the sum of thousands of group contributions per amplitude keeps FP32
// relative accuracy (FP64 accumulators add plainly).
template <typename R>
__device__ __forceinline__ void accumulate(V2<R> &acc, V2<R> &comp, R v, V2<R> p) {
    if constexpr (sizeof(R) == 4) {
        const R yx = v * p.x - comp.x;
        const R tx = acc.x + yx;
        comp.x = (tx - acc.x) - yx;
        acc.x = tx;
        const R yy = v * p.y - comp.y;
        const R ty = acc.y + yy;
        comp.y = (ty - acc.y) - yy;
        acc.y = ty;
    } else {
        acc.x += v * p.x;
        acc.y += v * p.y;
    }
}

// Fixed-order block sum (deterministic); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        s = (l < nw) ? red[l] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

// ---------------------------------------------------------------------------
// cos/sin of every schedule factor
// ---------------------------------------------------------------------------
template <typename R>
__global__ void cs_kernel(const double *__restrict__ theta, int K, const int32_t *__restrict__ op_k,
                          const double *__restrict__ op_scale, int n_ops, V2<R> *__restrict__ cs) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (o >= n_ops) return;
    double a = theta[(size_t)b * K + op_k[o]] * op_scale[o];
    double s, c;
    sincos(a, &s, &c);
    V2<R> v;
    v.x = (R)c;
    v.y = (R)s;
    cs[(size_t)b * n_ops + o] = v;
}

// ---------------------------------------------------------------------------
// Hamiltonian action and energy (Section 2.3): sigma = (H - shift) psi over
// X-mask groups.
//
// H conserves N_alpha and N_beta and psi vanishes outside the (n_alpha,
// n_beta) sector, so only sector amplitudes are read or produced.  A CTA
// owns one compact output tile: the sector amplitudes with fixed high bits
// h above the low LH bits, stored as a [C(LH/2, a)] x [C(LH/2, b)] array
// indexed by the ranks of their low alpha / beta strings (a, b = electrons
// the sector leaves for the low bits).  Each thread keeps up to kHEPT
// outputs in registers.  Groups are sorted into segments by the high part d
// of their X-mask; for each segment the compact source tile h ^ d is
// gathered into shared memory and every group of the segment adds
//   f_g(y) psi_y,  y = x ^ xmask_g,
// for the outputs whose flip pattern conserves the electron counts (then y
// lies in the source tile).  The own tile (d = 0) is the last segment, so
// psi_x is resident for the diagonal and the FP64 partials
// sum Re(conj(psi_x) sigma_x) and sum |psi_x|^2.  Entries of sigma outside
// the sector are never written (they stay zero).
// ---------------------------------------------------------------------------
constexpr int kHThreadsV = 256;
constexpr int kHEPT = 5;  // outputs per thread: 1280 >= C(7,3)^2, the largest 14-bit tile

struct HTileView {
    int a, b, Da, Db;
    const uint16_t *ca, *cb;  // low alpha / beta strings of the tile's class
};

__device__ __forceinline__ bool htile(const HSector &hs, int half, uint32_t hi, HTileView *v) {
    v->a = hs.n_alpha - __popc(hi & 0x55555555u);
    v->b = hs.n_beta - __popc(hi & 0xAAAAAAAAu);
    if (v->a < 0 || v->a > half || v->b < 0 || v->b > half) return false;
    const int32_t *o = hs.comb_offs + half * 17;
    v->Da = o[v->a + 1] - o[v->a];
    v->Db = o[v->b + 1] - o[v->b];
    v->ca = hs.combos + ((1 << half) - 1) + o[v->a];
    v->cb = hs.combos + ((1 << half) - 1) + o[v->b];
    return true;
}

template <typename R>
__global__ void __launch_bounds__(kHThreadsV) happly_kernel(const V2<R> *__restrict__ psi,
                                                            V2<R> *__restrict__ sig, size_t N,
                                                            int LH, DevHam<R> H, HSector hs,
                                                            double *__restrict__ Epart,
                                                            int store_sigma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *tile = reinterpret_cast<V2<R> *>(smem_raw);
    __shared__ double red[32];
    __shared__ uint32_t spa[1 << 8], spb[1 << 8];  // half-width string -> low bits
    __shared__ uint16_t rk[1 << 8];                 // rank of a half-width string
    const int b = blockIdx.y;
    const uint32_t h = blockIdx.x;
    const int half = LH >> 1;
    const V2<R> *src = psi + (size_t)b * N;
    for (int t = threadIdx.x; t < (1 << half); t += blockDim.x) {
        spa[t] = hs.spread[t];
        spb[t] = hs.spread[(1 << half) + t];
        rk[t] = hs.ranks[((1 << half) - 1) + t];
    }
    __syncthreads();
    HTileView ov;
    double e = 0.0, nrm = 0.0;
    if (htile(hs, half, h, &ov)) {
        const int D = ov.Da * ov.Db;
        uint32_t str[kHEPT];  // alpha string | beta string << 16, or ~0 when unused
        V2<R> acc[kHEPT], comp[kHEPT];
#pragma unroll
        for (int i = 0; i < kHEPT; ++i) {
            const int j = threadIdx.x + i * blockDim.x;
            if (j < D) {
                const int ia = j / ov.Db;
                str[i] = (uint32_t)ov.ca[ia] | ((uint32_t)ov.cb[j - ia * ov.Db] << 16);
            } else {
                str[i] = 0xFFFFFFFFu;
            }
            acc[i].x = acc[i].y = comp[i].x = comp[i].y = (R)0;
        }
        for (int s = 0; s < H.n_seg; ++s) {
            const uint32_t hsrc = h ^ H.seg_d[s];
            HTileView sv;
            if (!htile(hs, half, hsrc, &sv)) continue;  // source tile is all zero (uniform)
            const uint32_t base = hsrc << LH;
            const int Ds = sv.Da * sv.Db;
            __syncthreads();
            for (int j = threadIdx.x; j < Ds; j += blockDim.x) {
                const int ia = j / sv.Db;
                tile[j] = src[base | spa[sv.ca[ia]] | spb[sv.cb[j - ia * sv.Db]]];
            }
            __syncthreads();
            const int g_end = H.seg_begin[s + 1];
            for (int g = H.seg_begin[s]; g < g_end; ++g) {
                const GroupT<R> *G = H.groups + g;
                const uint32_t xm = G->xmask;
                const uint32_t jm = G->jmask;
                const uint32_t mla = G->mla, mlb = G->mlb;
                // occupied flip bits the source carries above the tile (uniform)
                const uint32_t xhi = xm >> LH;
                const int need_a = G->ha - __popc(hsrc & xhi & 0x55555555u);
                const int need_b = G->hb - __popc(hsrc & xhi & 0xAAAAAAAAu);
                const int nb = G->nb;
                const int spec = G->spec;
                const int p0 = G->pos[0], p1 = G->pos[1], p2 = G->pos[2], p3 = G->pos[3];
#pragma unroll
                for (int i = 0; i < kHEPT; ++i) {
                    if (str[i] == 0xFFFFFFFFu) continue;
                    const uint32_t ya = (str[i] & 0xFFFFu) ^ mla;
                    const uint32_t yb = (str[i] >> 16) ^ mlb;
                    if (__popc(ya & mla) != need_a || __popc(yb & mlb) != need_b) continue;
                    const uint32_t y = base | spa[ya] | spb[yb];
                    int pat = ((y >> p0) & 1u) | (((y >> p1) & 1u) << 1);
                    if (nb == 4) pat |= (((y >> p2) & 1u) << 2) | (((y >> p3) & 1u) << 3);
                    R v = G->lut[pat];
                    if (spec >= 0) {
                        uint32_t occ = y & ~xm;
                        while (occ) {
                            const int w = __ffs(occ) - 1;
                            occ &= occ - 1u;
                            v += H.spec[(size_t)(spec + w) * 4 + pat];
                        }
                    }
                    if (__popc(y & jm) & 1u) v = -v;
                    accumulate<R>(acc[i], comp[i], v, tile[rk[ya] * sv.Db + rk[yb]]);
                }
            }
        }
        // The last segment is the own tile (d = 0): psi_x is resident.
        const uint32_t own = h << LH;
        const int n = H.n;
#pragma unroll
        for (int i = 0; i < kHEPT; ++i) {
            if (str[i] == 0xFFFFFFFFu) continue;
            const uint32_t sa = str[i] & 0xFFFFu, sb = str[i] >> 16;
            const V2<R> p = tile[rk[sa] * ov.Db + rk[sb]];
            const uint32_t x = own | spa[sa] | spb[sb];
            if (H.has_diag) {
                long long q = H.diag_q0;
                uint32_t o1 = x;
                while (o1) {
                    const int a = __ffs(o1) - 1;
                    o1 &= o1 - 1u;
                    q += H.diag_qa[a];
                    uint32_t o2 = o1;
                    while (o2) {
                        const int r = __ffs(o2) - 1;
                        o2 &= o2 - 1u;
                        q += H.diag_qb[a * n + r];
                    }
                }
                accumulate<R>(acc[i], comp[i], (R)q * (R)H.diag_unit, p);
            }
            e += (double)p.x * (double)acc[i].x + (double)p.y * (double)acc[i].y;
            nrm += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            if (store_sigma) sig[(size_t)b * N + x] = acc[i];
        }
    }
    e = block_sum(e, red);
    nrm = block_sum(nrm, red);
    if (threadIdx.x == 0) {
        Epart[2 * ((size_t)b * gridDim.x + h)] = e;
        Epart[2 * ((size_t)b * gridDim.x + h) + 1] = nrm;
    }
}

// ---------------------------------------------------------------------------
// Final deterministic reductions: E[b] = sum over H tiles; grad[b][k] =
// sum over the schedule factors o of k of 2 * scale_o * sum over tiles.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) reduce_kernel(const double *__restrict__ Epart,
                                                          int n_tiles_h,
                                                          const double *__restrict__ gpart,
                                                          int tile_stride,
                                                          const int32_t *__restrict__ op_tiles,
                                                          int n_ops, int K,
                                                          const int32_t *__restrict__ k_ptr,
                                                          const int32_t *__restrict__ k_ops,
                                                          const double *__restrict__ op_scale,
                                                          double shift, int rayleigh,
                                                          double *__restrict__ E,
                                                          double *__restrict__ grad) {
    __shared__ double red[32];
    __shared__ double s_nrm;
    const int b = blockIdx.y;
    double e = 0.0, nr = 0.0;
    for (int t = threadIdx.x; t < n_tiles_h; t += blockDim.x) {
        e += Epart[2 * ((size_t)b * n_tiles_h + t)];
        nr += Epart[2 * ((size_t)b * n_tiles_h + t) + 1];
    }
    e = block_sum(e, red);
    nr = block_sum(nr, red);
    if (threadIdx.x == 0) {
        s_nrm = nr;
        if (blockIdx.x == 0) E[b] = rayleigh ? shift + e / nr : shift * nr + e;
    }
    __syncthreads();
    if (!grad) return;
    const double gscale = rayleigh ? 1.0 / s_nrm : 1.0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    for (int k = blockIdx.x * nw + warp; k < K; k += gridDim.x * nw) {
        double gk = 0.0;
        for (int u = k_ptr[k]; u < k_ptr[k + 1]; ++u) {
            const int o = k_ops[u];
            const double *p = gpart + ((size_t)b * n_ops + o) * tile_stride;
            const int nt = op_tiles[o];
            double s = 0.0;
            for (int t = lane; t < nt; t += 32) s += p[t];
            s = warp_sum(s);
            gk += 2.0 * op_scale[o] * s;
        }
        if (lane == 0) grad[(size_t)b * K + k] = gk * gscale;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
template <typename R>
size_t happly_smem(int max_entries) {
    return sizeof(V2<R>) * (size_t)max_entries;
}

template <typename R>
cudaError_t launch_cs(const LaunchCfg &cfg, const double *theta, int K, const int32_t *op_k,
                      const double *op_scale, void *cs) {
    dim3 grid((cfg.n_ops + kThreads - 1) / kThreads, cfg.B);
    cs_kernel<R><<<grid, kThreads, 0, cfg.stream>>>(theta, K, op_k, op_scale, cfg.n_ops,
                                                     static_cast<V2<R> *>(cs));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_happly(const LaunchCfg &cfg, const void *psi, void *sig, int LH,
                          const DevHam<R> &H, const HSector &hs, double *Epart, int store_sigma) {
    if (hs.max_entries > kHEPT * kHThreadsV) return cudaErrorInvalidValue;
    dim3 grid(1u << (cfg.n - LH), cfg.B);
    happly_kernel<R><<<grid, kHThreadsV, happly_smem<R>(hs.max_entries), cfg.stream>>>(
        static_cast<const V2<R> *>(psi), static_cast<V2<R> *>(sig), cfg.N, LH, H, hs, Epart,
        store_sigma);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const LaunchCfg &cfg, const double *Epart, int n_tiles_h,
                          const double *gpart, int tile_stride, const int32_t *op_tiles,
                          int K, const int32_t *k_ptr,
                          const int32_t *k_ops, const double *op_scale, double shift,
                          int rayleigh, double *E, double *grad) {
    int gx = grad ? std::max(1, std::min(64, (K + 7) / 8)) : 1;
    dim3 grid(gx, cfg.B);
    reduce_kernel<<<grid, kThreads, 0, cfg.stream>>>(Epart, n_tiles_h, gpart, tile_stride, op_tiles,
                                                     cfg.n_ops,
                                                     K, k_ptr, k_ops, op_scale, shift, rayleigh, E,
                                                     grad);
    return cudaGetLastError();
}

cudaError_t configure_kernels() {
    const int big = 200 * 1024;
    cudaError_t e;
#define UCCSD_SET(fn)                                                                  \
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, big);   \
    if (e != cudaSuccess) return e;
    UCCSD_SET((happly_kernel<float>));
    UCCSD_SET((happly_kernel<double>));
#undef UCCSD_SET
    return cudaSuccess;
}

#define UCCSD_INST(R)                                                                          \
    template size_t happly_smem<R>(int);                                                       \
    template cudaError_t launch_cs<R>(const LaunchCfg &, const double *, int, const int32_t *, \
                                      const double *, void *);                                 \
    template cudaError_t launch_happly<R>(const LaunchCfg &, const void *, void *, int,        \
                                          const DevHam<R> &, const HSector &, double *, int);
UCCSD_INST(float)
UCCSD_INST(double)
#undef UCCSD_INST

}  // namespace uccsd
