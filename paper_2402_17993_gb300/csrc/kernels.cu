// UCCSD state-vector kernels for GB300 (sm_103a).
//
// State layout: one slot = 2^n complex amplitudes (float2 or double2),
// slot b at offset b * 2^n; amplitude index x has bit P = occupation of
// spin orbital P.  Nothing here is a dense contraction, so no tensor cores:
// the rotations are bandwidth bound, the Hamiltonian action is ALU bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "amp.cuh"
#include "kernels.cuh"
#include "pdl.cuh"

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
    if constexpr (sizeof(R) == 4) {
        // the FP32 rotation takes d = 1 - cos = 2 sin^2(a / 2), exact to FP32
        // rounding for small angles (1 - cos would cancel)
        const double h = sin(0.5 * a);
        v.x = (R)(2.0 * h * h);
    } else {
        v.x = (R)c;
    }
    v.y = (R)s;
    cs[(size_t)b * n_ops + o] = v;
}

// ---------------------------------------------------------------------------
// Hamiltonian action and energy (Section 2.3): sigma = (H - shift) psi,
// accumulated over the X-mask groups of the Jordan-Wigner Hamiltonian.
//
// H conserves N_alpha and N_beta, and psi vanishes outside the (n_alpha,
// n_beta) sector, so every output and every source is a sector amplitude,
// written x = (alpha string, beta string).  A CTA owns a block of columns
// (beta strings, one per lane and slot) of one row (alpha string R).  For
// output x the groups with a nonzero contribution are exactly those whose
// flip connects x to a sector source y = x ^ xmask_g, so the CTA visits them
// by class instead of testing all groups:
//   - the diagonal group (occupation quadratic form, 64-bit fixed point);
//   - beta-only groups from the own row: each lane enumerates the beta
//     single (j -> b) and double (j1 j2 -> b1 b2) excitations of its column;
//   - for every alpha single excitation p -> q of R the source row
//     R ^ {p, q} is gathered into shared memory; the alpha-only pair group
//     acts column-wise and the mixed groups (alpha pair, beta pair) through
//     each lane's beta single excitations;
//   - for every alpha double excitation of R the alpha-only quad group reads
//     the source amplitude of the same column directly.
// Every lane runs the same loop trip counts (its column has n_beta
// electrons), so the warps do not diverge.  The contribution of group g is
// f_g(y) psi_y with f_g(y) = (-1)^{popc(y & J_g)} (LUT_g[pattern of y] +
// sum of the spectator rows of y's other occupied orbitals).  FP32
// accumulators are Kahan-compensated.  The FP64 partials sum Re(conj(psi_x)
// sigma_x) and sum |psi_x|^2 feed the energy; sigma outside the sector is
// never written (it stays zero).
// ---------------------------------------------------------------------------
// Dynamic shared memory of the H-apply: one source row, the beta string
// ranks, then (16-byte aligned) the row's beta-single values.
template <typename R>
__host__ __device__ inline size_t happly_aspec_offset(int Db, int n_orb) {
    const size_t o = sizeof(V2<R>) * (size_t)Db + sizeof(uint16_t) * ((size_t)1 << n_orb);
    return (o + 15) & ~(size_t)15;
}

// Row part of a beta single j -> b (pair group pb, source side sel), entry
// 2 pb + sel: the table value plus the alpha-spectator sum of the row, and
// the row's part of the Jordan-Wigner sign (bit 31: the parities of the
// row's occupied alpha orbitals up to j and up to b).
template <typename R>
struct alignas(2 * sizeof(R) > 8 ? 16 : 8) RowB {
    R v;
    uint32_t s;
};

// One alpha single excitation of an H-apply row: source alpha string,
// source row offset, p | q << 8 (p occupied, q empty in the target).
struct ASgl {
    uint32_t s, xoff, pq;
};

// Shared-memory layout after the aspec block (offsets 16-byte aligned):
// the row's alpha singles, its alpha doubles, then for a phase of G alpha
// singles their source rows ([column][G]; see item_value),
// their rows of the ordered mixed table with the row's signs folded in
// ([j * n_orb + b][G], then the same negated) and their alpha-only values; last, while the CTA stays within
// kHappBbStage bytes, a copy of the signed beta-double table (dbt = 0: the
// kernel reads it from global memory).
struct HappLayout {
    size_t asl, adl, srcg, mrow, asing, dbt, total;
};
constexpr size_t kHappBbStage = 32 * 1024;
template <typename R>
__host__ __device__ inline HappLayout happly_layout(int Db, int n_orb, int n_alpha, int G) {
    auto up = [](size_t o) { return (o + 15) & ~(size_t)15; };
    const int nva = n_orb - n_alpha;
    const size_t nas = (size_t)n_alpha * nva;
    const size_t nad = (size_t)(n_alpha * (n_alpha - 1) / 2) * (nva * (nva - 1) / 2);
    HappLayout L;
    L.asl = up(happly_aspec_offset<R>(Db, n_orb) + sizeof(RowB<R>) * (size_t)n_orb * (n_orb - 1));
    L.adl = up(L.asl + sizeof(ASgl) * nas);
    L.srcg = up(L.adl + sizeof(ADbl<R>) * nad);
    L.mrow = up(L.srcg + sizeof(V2<R>) * (size_t)G * Db);
    L.asing = up(L.mrow + sizeof(R) * (size_t)2 * G * n_orb * n_orb);
    L.total = L.asing + sizeof(R) * (size_t)G;
    const size_t np = (size_t)n_orb * (n_orb - 1) / 2;
    const size_t bb = up(L.total);
    L.dbt = 0;
    if (bb + sizeof(R) * np * np <= kHappBbStage) {
        L.dbt = bb;
        L.total = bb + sizeof(R) * np * np;
    }
    return L;
}

// Bit v = parity of the bits 0 .. v of x (16-bit strings).
__device__ __forceinline__ uint32_t prefix_parity(uint32_t x) {
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    return x;
}

__device__ __forceinline__ int pair_index(int p, int q) {  // p < q
    return (q * (q - 1) >> 1) + p;
}

// Sign bit (bit 31) of the Jordan-Wigner parity of a group with mask j (alpha
// bits low, beta bits high) at the source strings packed as ya | yb << 16.
__device__ __forceinline__ uint32_t jw_sign(uint32_t packed, uint32_t j) {
    return (uint32_t)__popc(packed & j) << 31;
}
__device__ __forceinline__ float with_sign(float x, uint32_t s) {
    return __int_as_float(__float_as_int(x) ^ (int)(s & 0x80000000u));
}
__device__ __forceinline__ double with_sign(double x, uint32_t s) {
    return __hiloint2double(__double2hiint(x) ^ (int)(s & 0x80000000u), __double2loint(x));
}


// Shared-memory arrays of n items of AG values of type T.  With CH set, an
// item of more than 16 bytes is stored as 16-byte chunks, chunk k of every
// item before chunk k + 1 ([k][item]), so that a warp's 16-byte loads of
// random items fall on all eight 16-byte bank groups; otherwise (and for
// items of 16 bytes or less) items are stored plainly, [item][value].
// Measured on the FP32 H-apply's staged source rows (32-byte items):
// chunks at one column per thread (18 qubits, 126 columns: 0.494 -> 0.455
// ms), plain at eight columns per thread (26 qubits, 1716 columns: chunks
// 8.17 against 7.48 ms).  Value g of item i:
template <typename T, int AG, bool CH>
__device__ __forceinline__ T *item_value(void *base, int n, int i, int g) {
    constexpr int B = int(sizeof(T)) * AG;
    unsigned char *p = static_cast<unsigned char *>(base);
    if constexpr (B <= 16 || !CH) {
        return reinterpret_cast<T *>(p + (size_t)i * B) + g;
    } else {
        const int byte = g * (int)sizeof(T);
        return reinterpret_cast<T *>(p + ((size_t)(byte >> 4) * n + i) * 16 + (byte & 15));
    }
}
// All AG values of item i, in 16-byte (or one 8- or 4-byte) loads.
template <typename T, int AG, bool CH>
__device__ __forceinline__ void item_load(const void *base, int n, int i, T (&v)[AG]) {
    constexpr int B = int(sizeof(T)) * AG;
    const unsigned char *p = static_cast<const unsigned char *>(base);
    if constexpr (B > 16) {
        int4 w[B / 16];
#pragma unroll
        for (int k = 0; k < B / 16; ++k)
            w[k] = *reinterpret_cast<const int4 *>(p + (CH ? ((size_t)k * n + i) * 16 : (size_t)i * B + 16 * k));
        __builtin_memcpy(&v[0], &w[0], B);
    } else if constexpr (B == 16) {
        const int4 w = *reinterpret_cast<const int4 *>(p + (size_t)i * 16);
        __builtin_memcpy(&v[0], &w, 16);
    } else if constexpr (B == 8) {
        const int2 w = *reinterpret_cast<const int2 *>(p + (size_t)i * 8);
        __builtin_memcpy(&v[0], &w, 8);
    } else {
        v[0] = *reinterpret_cast<const T *>(p + (size_t)i * B);
    }
}

// The alpha singles p -> q of row R, AG per phase (source rows R ^ {p, q}):
// the alpha-only pair group of each single on the lane's own column, and
// the mixed groups (alpha pair, beta pair) through the lane's beta single
// excitations j -> b.
//
// Sign of a mixed contribution.  The group's Jordan-Wigner mask is the
// interval mask of its flipped qubits 2p, 2q (alpha) and 2j + 1, 2b + 1
// (beta): the XOR of the bit masks below each, without the flipped bits.
// Over beta orbitals that is (A_pq ^ B_jb) minus {j, b}, with A_pq =
// L(p) ^ L(q), B_jb = L(j) ^ L(b) and L(v) the bits below v.  The source
// beta string equals the column's string s_c except at j (occupied in s_c)
// and b (empty), so the source's parity under the mask splits into
//   popc(s_c & A_pq)                       column x alpha single,
//   bit j of A_pq, and the alpha part      alpha single x (j, b),
//   s_c's occupied orbitals strictly between j and b   column x beta single.
// The middle term is folded into the staged table, the last one selects the
// table's negated half (HSector::bmix), and the first flips the single's
// partial sum once.  Sign flips are exact, so every partial sum equals,
// bit for bit, the one formed with a sign per term.
template <typename R, int EPT, int AG>
__device__ __forceinline__ void alpha_phases(const V2<R> *__restrict__ st, const DevHam<R> &H,
                                             const HSector &hs, const ASgl *asl, V2<R> *srcg,
                                             R *tw, R *asing, const int (&cix)[EPT],
                                             const uint32_t (&sc)[EPT], V2<R> (&acc)[EPT],
                                             V2<R> (&comp)[EPT]) {
    constexpr bool CH = EPT == 1;  // chunked staged arrays (see item_value)
    const int n_orb = H.n_orb;
    const int nas = hs.n_alpha * (n_orb - hs.n_alpha);
    const int nn = n_orb * n_orb;
    for (int g0 = 0; g0 < nas; g0 += AG) {
        const int gn = min(AG, nas - g0);
        __syncthreads();  // the previous phase's rows are consumed
        for (int t = threadIdx.x; t < hs.Db * AG; t += blockDim.x) {
            const int c = t / AG, g = t % AG;
            V2<R> v = V2<R>{(R)0, (R)0};
            if (g < gn) v = st[asl[g0 + g].xoff + hs.boff[hs.bstr[c]]];
            *item_value<V2<R>, AG, CH>(srcg, hs.Db, c, g) = v;
        }
        for (int t = threadIdx.x; t < nn * AG; t += blockDim.x) {
            const int jb = t / AG, g = t % AG;
            R w = (R)0;
            if (g < gn) {
                const ASgl a = asl[g0 + g];
                const int p = (int)(a.pq & 0xFFu), q = (int)(a.pq >> 8);
                const MixO<R> M = H.mixo[(size_t)(p * n_orb + q) * nn + jb];
                const uint32_t apq = ((1u << p) - 1u) ^ ((1u << q) - 1u);
                const uint32_t par = (uint32_t)__popc(a.s & M.j & 0xFFFFu) ^ (apq >> (jb / n_orb));
                w = with_sign(M.w, par << 31);
            }
            *item_value<R, AG, CH>(tw, 2 * nn, jb, g) = w;
            *item_value<R, AG, CH>(tw, 2 * nn, nn + jb, g) = with_sign(w, 0x80000000u);
        }
        if (threadIdx.x < gn) {
            // the alpha-only group value's alpha part: the same for every column
            const ASgl a = asl[g0 + threadIdx.x];
            const int p = (int)(a.pq & 0xFFu), q = (int)(a.pq >> 8);
            const int asel = q > p;
            const SglT<R> &S = H.s1a[pair_index(min(p, q), max(p, q))];
            R va = S.lut[asel];
            if (S.spec >= 0)
                for (uint32_t w = a.s & ~(1u << q); w; w &= w - 1u)
                    va += H.spec[(size_t)(S.spec + 2 * (__ffs(w) - 1)) * 4 + (asel ? 2 : 1)];
            asing[threadIdx.x] = va;
        }
        __syncthreads();
        uint32_t apq[AG];
#pragma unroll
        for (int g = 0; g < AG; ++g) {
            const uint32_t pq = g < gn ? asl[g0 + g].pq : 0u;
            apq[g] = ((1u << (pq & 0xFFu)) - 1u) ^ ((1u << (pq >> 8)) - 1u);
        }
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            if (cix[i] < 0) continue;
            const uint32_t cb_str = sc[i];
            // one table entry and one source entry per beta single serve the
            // phase's AG alpha singles: a plain partial sum per alpha single,
            // added with compensation
            V2<R> seg[AG];
#pragma unroll
            for (int g = 0; g < AG; ++g) seg[g] = V2<R>{(R)0, (R)0};
            const uint32_t *bm = hs.bmix + cix[i];
#pragma unroll 2
            for (int t = 0; t < hs.n_bs; ++t) {
                const uint32_t e = __ldg(bm + (size_t)t * hs.Db);
                R w[AG];
                V2<R> y[AG];
                item_load<R, AG, CH>(tw, 2 * nn, (int)(e >> 16), w);
                item_load<V2<R>, AG, CH>(srcg, hs.Db, (int)(e & 0xFFFFu), y);
#pragma unroll
                for (int g = 0; g < AG; ++g) {
                    seg[g].x += w[g] * y[g].x;
                    seg[g].y += w[g] * y[g].y;
                }
            }
#pragma unroll
            for (int g = 0; g < AG; ++g) {
                if (g < gn) {
                    const ASgl a = asl[g0 + g];
                    const int p = (int)(a.pq & 0xFFu), q = (int)(a.pq >> 8);
                    const int pa = pair_index(min(p, q), max(p, q));
                    const int asel = q > p;
                    // alpha-only pair group: same column (beta-spectator sum per column)
                    R val = asing[g] + __ldg(H.bspec_a + ((size_t)pa * 2 + asel) * hs.Db + cix[i]);
                    val = with_sign(val, jw_sign(a.s | (cb_str << 16), H.s1a[pa].j));
                    accumulate<R>(acc[i], comp[i], val, *item_value<V2<R>, AG, CH>(srcg, hs.Db, cix[i], g));
                    accumulate<R>(acc[i], comp[i], (__popc(cb_str & apq[g]) & 1) ? (R)-1 : (R)1,
                                  seg[g]);
                }
            }
        }
    }
}

template <typename R, int EPT>
__global__ void __launch_bounds__(kRowThreads) happly_kernel(const V2<R> *__restrict__ psi,
                                                             V2<R> *__restrict__ sig, size_t N,
                                                             DevHam<R> H, HSector hs,
                                                             double *__restrict__ Epart,
                                                             int flags) {
    pdl_wait();  // psi is the previous kernel's output
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *src = reinterpret_cast<V2<R> *>(smem_raw);                  // one source row
    uint16_t *brk = reinterpret_cast<uint16_t *>(src + hs.Db);          // beta string ranks
    // row part of each beta single, [pair][sel]
    RowB<R> *rowb = reinterpret_cast<RowB<R> *>(smem_raw + happly_aspec_offset<R>(hs.Db, H.n_orb));
    const HappLayout lay = happly_layout<R>(hs.Db, H.n_orb, hs.n_alpha, hs.ag);
    ASgl *asl = reinterpret_cast<ASgl *>(smem_raw + lay.asl);
    ADbl<R> *adl = reinterpret_cast<ADbl<R> *>(smem_raw + lay.adl);
    V2<R> *srcg = reinterpret_cast<V2<R> *>(smem_raw + lay.srcg);
    R *tw = reinterpret_cast<R *>(smem_raw + lay.mrow);
    R *asing = reinterpret_cast<R *>(smem_raw + lay.asing);
    __shared__ double red[32];
    __shared__ int nb4[16 * 5];
    __shared__ long long xrow[16];  // diagonal: row's alpha-beta pair sums per beta orbital
    __shared__ long long qrow;      // diagonal: constant plus the row's alpha part
    const int b = blockIdx.y;
    const int row = blockIdx.x / hs.ncb;
    const int cb = blockIdx.x - row * hs.ncb;
    const int n_orb = H.n_orb;
    const uint32_t full = (1u << n_orb) - 1u;
    const uint32_t sR = hs.astr[row];
    const V2<R> *st = psi + (size_t)b * N;
    for (int t = threadIdx.x; t < (1 << n_orb); t += blockDim.x) brk[t] = hs.brank[t];
    for (int t = threadIdx.x; t < 16 * 5; t += blockDim.x) nb4[t] = hs.binom[t];
    // parity of the row's occupied alpha orbitals up to v, bit v
    const uint32_t pa = prefix_parity(sR);
    for (int t = threadIdx.x; t < 2 * H.n_pairs; t += blockDim.x) {
        const SglT<R> &S = H.s1b[t >> 1];
        R val = (R)0;
        if (S.spec >= 0) {
            const int pat = (t & 1) ? 2 : 1;
            for (uint32_t w = sR; w; w &= w - 1u)
                val += H.spec[(size_t)(S.spec + 2 * (__ffs(w) - 1)) * 4 + pat];
        }
        int hi = 1;
        while ((hi + 1) * hi / 2 <= (t >> 1)) ++hi;
        const int lo = (t >> 1) - hi * (hi - 1) / 2;
        RowB<R> rb;
        rb.v = S.lut[t & 1] + val;
        rb.s = ((pa >> lo) ^ (pa >> hi)) << 31;
        rowb[t] = rb;
    }
    const int np = H.n_pairs;
    const R *dbt = H.d2bs;
    if (lay.dbt) {
        R *d = reinterpret_cast<R *>(smem_raw + lay.dbt);
        for (int t = threadIdx.x; t < np * np; t += blockDim.x) d[t] = __ldg(H.d2bs + t);
        dbt = d;
    }
    {
        const uint32_t xR = hs.aoff[sR];
        for (int c = threadIdx.x; c < hs.Db; c += blockDim.x)
            src[c] = st[xR + hs.boff[hs.bstr[c]]];
    }
    // the row's alpha singles in loop order (p occupied ascending, then q
    // empty ascending): entry ip * nva + iq
    const uint32_t virA = full & ~sR;
    for (int t = threadIdx.x; t < hs.n_alpha * (n_orb - hs.n_alpha); t += blockDim.x) {
        const int nv = n_orb - hs.n_alpha;
        int ip = t / nv, iq = t - (t / nv) * nv;
        uint32_t o = sR, v = virA;
        for (; ip > 0; --ip) o &= o - 1u;
        for (; iq > 0; --iq) v &= v - 1u;
        const int p = __ffs(o) - 1, q = __ffs(v) - 1;
        const uint32_t sRp = sR ^ (1u << p) ^ (1u << q);
        ASgl a;
        a.s = sRp;
        a.xoff = hs.aoff[sRp];
        a.pq = (uint32_t)p | ((uint32_t)q << 8);
        asl[t] = a;
    }
    // the row's alpha doubles: occupied pair t (loop order o1 < o2) owns the
    // entries [t * nvp, (t + 1) * nvp) over the empty pairs (q1 < q2)
    const int nva = n_orb - hs.n_alpha;
    const int nop = hs.n_alpha * (hs.n_alpha - 1) / 2, nvp = nva * (nva - 1) / 2;
    for (int t = threadIdx.x; t < nop; t += blockDim.x) {
        int k = 0, p1 = -1, p2 = -1;
        for (uint32_t o1 = sR; o1 && p1 < 0; o1 &= o1 - 1u)
            for (uint32_t o2 = o1 & (o1 - 1u); o2; o2 &= o2 - 1u, ++k)
                if (k == t) {
                    p1 = __ffs(o1) - 1;
                    p2 = __ffs(o2) - 1;
                    break;
                }
        const MixO<R> *Dp = H.d2ao + (size_t)(p1 * n_orb + p2) * n_orb * n_orb;
        ADbl<R> *L = adl + (size_t)t * nvp;
        int m = 0;
        for (uint32_t v1 = virA; v1; v1 &= v1 - 1u) {
            const int q1 = __ffs(v1) - 1;
            for (uint32_t v2 = v1 & (v1 - 1u); v2; v2 &= v2 - 1u) {
                const int q2 = __ffs(v2) - 1;
                const MixO<R> Dq = Dp[q1 * n_orb + q2];
                const uint32_t sRp = sR ^ ((1u << p1) | (1u << p2) | (1u << q1) | (1u << q2));
                ADbl<R> e;
                e.w = Dq.w;
                e.xoff = hs.aoff[sRp];
                e.s = sRp;
                e.j = Dq.j;
                L[m++] = e;
            }
        }
    }
    if (H.has_diag) {
        // alpha orbital i is qubit 2i, beta orbital j qubit 2j + 1
        const int t = blockDim.x > 96 ? (int)threadIdx.x - 64 : (int)threadIdx.x;
        if (t >= 0 && t < n_orb) {
            const int r = 2 * t + 1;
            long long v = 0;
            for (uint32_t w = sR; w; w &= w - 1u) {
                const int a = 2 * (__ffs(w) - 1);
                v += H.diag_qb[(size_t)min(a, r) * H.n + max(a, r)];
            }
            xrow[t] = v;
        } else if (t == n_orb) {
            long long v = H.diag_q0;
            for (uint32_t w = sR; w; w &= w - 1u) {
                const int a = 2 * (__ffs(w) - 1);
                v += H.diag_qa[a];
                for (uint32_t w2 = w & (w - 1u); w2; w2 &= w2 - 1u)
                    v += H.diag_qb[(size_t)a * H.n + 2 * (__ffs(w2) - 1)];
            }
            qrow = v;
        }
    }
    __syncthreads();

    int cix[EPT];
    uint32_t sc[EPT];
    V2<R> acc[EPT], comp[EPT], own[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        const int loc = threadIdx.x + i * blockDim.x;
        const int c = cb * hs.colblock + loc;
        cix[i] = (loc < hs.colblock && c < hs.Db) ? c : -1;
        sc[i] = cix[i] >= 0 ? hs.bstr[c] : 0u;
        own[i] = cix[i] >= 0 ? src[c] : V2<R>{(R)0, (R)0};
        acc[i] = V2<R>{(R)0, (R)0};
        comp[i] = V2<R>{(R)0, (R)0};
    }

    // ---- own row: diagonal, beta singles, beta doubles ----
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        if (cix[i] < 0) continue;
        const uint32_t cb_str = sc[i];
        if (H.has_diag) {
            // the occupation form over all occupied qubits: the row's part,
            // the column's beta part and the alpha-beta pairs (exact integers)
            long long q = qrow + __ldg(H.diag_col + cix[i]);
            for (uint32_t w = cb_str; w; w &= w - 1u) q += xrow[__ffs(w) - 1];
            accumulate<R>(acc[i], comp[i], (R)q * (R)H.diag_unit, own[i]);
        }
        // Jordan-Wigner signs of the beta-only groups from prefix parities:
        // for a beta excitation the group's mask over alpha orbitals is the
        // XOR of "up to v" masks and over beta orbitals the XOR of "below v"
        // masks, v over its orbitals, without the flipped bits; so its sign
        // is the XOR of bit v of pa ^ pb over those orbitals and a term of
        // the excitation alone (in the tables)
        const uint32_t pab = pa ^ prefix_parity(cb_str << 1);
        // beta singles (precomputed per column: source rank, row-table
        // entry, column sign, beta-spectator sum)
        {
            const uint2 *bsc = hs.bsing + cix[i];
            const R *bsp = H.bspec_b + cix[i];
            for (int t = 0; t < hs.n_bs; ++t) {
                const uint2 e = __ldg(bsc + (size_t)t * hs.Db);
                const RowB<R> rb = rowb[e.y >> 16];
                R val = rb.v + __ldg(bsp + (size_t)t * hs.Db);
                val = with_sign(val, rb.s ^ (e.y << 31));
                accumulate<R>(acc[i], comp[i], val, src[e.x & 0xFFFFu]);
            }
        }
        const uint32_t vir = full & ~cb_str;
        for (uint32_t o1 = cb_str; o1; o1 &= o1 - 1u) {
            const int j1 = __ffs(o1) - 1;
            for (uint32_t o2 = o1 & (o1 - 1u); o2; o2 &= o2 - 1u) {
                const int j2 = __ffs(o2) - 1;
                const R *Dj = dbt + (size_t)pair_index(j1, j2) * np;
                const uint32_t yj = cb_str ^ (1u << j1) ^ (1u << j2);
                const uint32_t s12 = (pab >> j1) ^ (pab >> j2);
                V2<R> seg = V2<R>{(R)0, (R)0};  // plain partial per occupied pair
                for (uint32_t v1 = vir; v1; v1 &= v1 - 1u) {
                    const int b1 = __ffs(v1) - 1;
                    const uint32_t y1 = yj ^ (1u << b1);
                    const uint32_t s1 = s12 ^ (pab >> b1);
                    for (uint32_t v2 = v1 & (v1 - 1u); v2; v2 &= v2 - 1u) {
                        const int b2 = __ffs(v2) - 1;
                        const R val = with_sign(Dj[pair_index(b1, b2)], (s1 ^ (pab >> b2)) << 31);
                        const V2<R> y = src[brk[y1 ^ (1u << b2)]];
                        seg.x += val * y.x;
                        seg.y += val * y.y;
                    }
                }
                accumulate<R>(acc[i], comp[i], (R)1, seg);
            }
        }
    }

    // ---- alpha singles, hs.ag per phase: source rows R ^ {p, q} ----
    switch (hs.ag) {
        case 4: alpha_phases<R, EPT, 4>(st, H, hs, asl, srcg, tw, asing, cix, sc, acc, comp); break;
        case 2: alpha_phases<R, EPT, 2>(st, H, hs, asl, srcg, tw, asing, cix, sc, acc, comp); break;
        default: alpha_phases<R, EPT, 1>(st, H, hs, asl, srcg, tw, asing, cix, sc, acc, comp); break;
    }

    // ---- alpha doubles: source amplitude of the same column ----
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        if (cix[i] < 0) continue;
        const uint32_t boffc = hs.boff[sc[i]];
        const uint32_t cbs = sc[i] << 16;
        for (int t = 0; t < nop; ++t) {
            const ADbl<R> *L = adl + (size_t)t * nvp;
            V2<R> dseg = V2<R>{(R)0, (R)0};  // plain partial per occupied pair
#pragma unroll 4
            for (int m = 0; m < nvp; ++m) {
                const ADbl<R> e = L[m];
                const R val = with_sign(e.w, jw_sign(e.s | cbs, e.j));
                const V2<R> y = st[e.xoff + boffc];
                dseg.x += val * y.x;
                dseg.y += val * y.y;
            }
            accumulate<R>(acc[i], comp[i], (R)1, dseg);
        }
    }

    double e = 0.0, nrm = 0.0;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        if (cix[i] < 0) continue;
        const V2<R> p = own[i];
        V2<R> out = acc[i];
        if (sizeof(R) == 8 || (flags & kHApplyComplex32)) {
            e += amp::re_dot(p, out);
            nrm += amp::re_dot(p, p);
        } else {
            // FP32 state, real amplitudes as hi + lo: the Kahan terms of both
            // words join lo (true sum = acc - comp)
            out.y = out.y - comp[i].y - comp[i].x;
            const double pv = (double)p.x + (double)p.y;
            e += pv * ((double)out.x + (double)out.y);
            nrm += pv * pv;
        }
        if (flags & kHApplyStoreSigma) sig[(size_t)b * N + (hs.aoff[sR] + hs.boff[sc[i]])] = out;
    }
    e = block_sum(e, red);
    nrm = block_sum(nrm, red);
    if (threadIdx.x == 0) {
        Epart[2 * ((size_t)b * gridDim.x + blockIdx.x)] = e;
        Epart[2 * ((size_t)b * gridDim.x + blockIdx.x) + 1] = nrm;
    }
}

// Energy of slot b from the H-apply's tile partials, summed by the first
// warp in a fixed order (the same in every reduction kernel, so energy-only
// and energy+gradient calls agree bitwise); the norm goes to *s_nrm.
__device__ __forceinline__ void energy_sums(const double *__restrict__ Epart, int n_tiles_h, int b,
                                            double shift, int rayleigh, double *__restrict__ E,
                                            double *s_nrm) {
    if (threadIdx.x >= 32) return;
    double e = 0.0, nr = 0.0;
    for (int t = threadIdx.x; t < n_tiles_h; t += 32) {
        e += Epart[2 * ((size_t)b * n_tiles_h + t)];
        nr += Epart[2 * ((size_t)b * n_tiles_h + t) + 1];
    }
    e = warp_sum(e);
    nr = warp_sum(nr);
    if (threadIdx.x == 0) {
        *s_nrm = nr;
        if (blockIdx.x == 0) E[b] = rayleigh ? shift + e / nr : shift * nr + e;
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
    pdl_wait();  // the partials are the previous kernels' output
    __shared__ double s_nrm;
    const int b = blockIdx.y;
    energy_sums(Epart, n_tiles_h, b, shift, rayleigh, E, &s_nrm);
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

// The same reductions with one thread per gradient component, for plans
// whose factors have few partial slots (the pair-list adjoint writes one per
// tile and warp: 32 at 18 qubits).  GB300's FP64 rate is low, so the energy
// and norm are summed by one warp per block instead of a block-wide tree in
// every block, and each component's partials by one thread in slot order.
constexpr int kReduceSerialMax = 64;

__global__ void __launch_bounds__(kThreads) reduce_serial_kernel(
    const double *__restrict__ Epart, int n_tiles_h, const double *__restrict__ gpart,
    int tile_stride, const int32_t *__restrict__ op_tiles, int n_ops, int K,
    const int32_t *__restrict__ k_ptr, const int32_t *__restrict__ k_ops,
    const double *__restrict__ op_scale, double shift, int rayleigh, double *__restrict__ E,
    double *__restrict__ grad) {
    __shared__ double s_nrm;
    const int b = blockIdx.y;
    energy_sums(Epart, n_tiles_h, b, shift, rayleigh, E, &s_nrm);
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double gscale = rayleigh ? 1.0 / s_nrm : 1.0;
    double gk = 0.0;
    for (int u = k_ptr[k]; u < k_ptr[k + 1]; ++u) {
        const int o = k_ops[u];
        const double *p = gpart + ((size_t)b * n_ops + o) * tile_stride;
        const int nt = op_tiles[o];
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += p[t];
        gk += 2.0 * op_scale[o] * s;
    }
    grad[(size_t)b * K + k] = gk * gscale;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Fixed-step L-BFGS update on the device (two-loop recursion, Nocedal and
// Wright Algorithm 7.4), one CTA: the serving loop's optimiser step without
// a host round trip.  State (all device): S, Y [m][K] ring of (s, y) pairs,
// rho [m], prev_theta, prev_g, work [K], meta = {count, head, has_prev,
// step}.  Pairs with s.y <= 1e-16 max(1, y.y) are not stored; the step is
// -first_scale g while no pair is stored; the step is capped at max_step in
// the max-norm.  All dot products are FP64 in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kOptThreads = 256;

__device__ double opt_dot(const double *a, const double *b, int K, double *red) {
    double v = 0.0;
    for (int i = threadIdx.x; i < K; i += kOptThreads) v += a[i] * b[i];
    v = block_sum(v, red);
    __shared__ double bc;
    if (threadIdx.x == 0) bc = v;
    __syncthreads();
    v = bc;
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(kOptThreads) lbfgs_kernel(
    int K, int m, double max_step, double first_scale, double *__restrict__ theta,
    const double *__restrict__ E, const double *__restrict__ g, double *__restrict__ S,
    double *__restrict__ Y, double *__restrict__ rho, double *__restrict__ prev_t,
    double *__restrict__ prev_g, double *__restrict__ work, int *__restrict__ meta,
    double *__restrict__ E_hist, int max_steps) {
    __shared__ double red[32];
    __shared__ double alpha[64];
    const int count0 = meta[0], head0 = meta[1], has_prev = meta[2], step = meta[3];
    if (threadIdx.x == 0 && step < max_steps) E_hist[step] = E[0];
    int count = count0, head = head0;
    if (has_prev) {
        const int nxt = (head0 + 1) % m;
        double *sn = S + (size_t)nxt * K, *yn = Y + (size_t)nxt * K;
        for (int i = threadIdx.x; i < K; i += kOptThreads) {
            sn[i] = theta[i] - prev_t[i];
            yn[i] = g[i] - prev_g[i];
        }
        __syncthreads();
        const double sy = opt_dot(sn, yn, K, red);
        const double yy = opt_dot(yn, yn, K, red);
        if (sy > 1e-16 * fmax(1.0, yy)) {
            if (threadIdx.x == 0) rho[nxt] = 1.0 / sy;
            head = nxt;
            count = min(count0 + 1, m);
        }
        __syncthreads();
    }
    // direction d in work
    if (count == 0) {
        for (int i = threadIdx.x; i < K; i += kOptThreads) work[i] = -first_scale * g[i];
        __syncthreads();
    } else {
        for (int i = threadIdx.x; i < K; i += kOptThreads) work[i] = g[i];
        __syncthreads();
        for (int k = 0; k < count; ++k) {  // newest first
            const int idx = (head - k + m) % m;
            const double a = rho[idx] * opt_dot(S + (size_t)idx * K, work, K, red);
            if (threadIdx.x == 0) alpha[k] = a;
            for (int i = threadIdx.x; i < K; i += kOptThreads) work[i] -= a * Y[(size_t)idx * K + i];
            __syncthreads();
        }
        const double *yh = Y + (size_t)head * K, *sh = S + (size_t)head * K;
        const double gamma = opt_dot(sh, yh, K, red) / opt_dot(yh, yh, K, red);
        for (int i = threadIdx.x; i < K; i += kOptThreads) work[i] *= gamma;
        __syncthreads();
        for (int k = count - 1; k >= 0; --k) {  // oldest first
            const int idx = (head - k + m) % m;
            const double b = rho[idx] * opt_dot(Y + (size_t)idx * K, work, K, red);
            const double c = alpha[k] - b;
            for (int i = threadIdx.x; i < K; i += kOptThreads) work[i] += c * S[(size_t)idx * K + i];
            __syncthreads();
        }
        for (int i = threadIdx.x; i < K; i += kOptThreads) work[i] = -work[i];
        __syncthreads();
    }
    // cap in the max-norm
    double mx = 0.0;
    for (int i = threadIdx.x; i < K; i += kOptThreads) mx = fmax(mx, fabs(work[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kOptThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) alpha[63] = v;
    }
    __syncthreads();
    mx = alpha[63];
    const double scale = mx > max_step ? max_step / mx : 1.0;
    for (int i = threadIdx.x; i < K; i += kOptThreads) {
        prev_t[i] = theta[i];
        prev_g[i] = g[i];
        theta[i] += work[i] * scale;
    }
    if (threadIdx.x == 0) {
        meta[0] = count;
        meta[1] = head;
        meta[2] = 1;
        meta[3] = step + 1;
    }
}

cudaError_t launch_lbfgs(cudaStream_t stream, int K, int m, double max_step, double first_scale,
                         double *theta, const double *E, const double *g, double *state,
                         int *meta, double *E_hist, int max_steps) {
    double *S = state, *Y = S + (size_t)m * K, *rho = Y + (size_t)m * K;
    double *prev_t = rho + m, *prev_g = prev_t + K, *work = prev_g + K;
    lbfgs_kernel<<<1, kOptThreads, 0, stream>>>(K, m, max_step, first_scale, theta, E, g, S, Y, rho,
                                                prev_t, prev_g, work, meta, E_hist, max_steps);
    return cudaGetLastError();
}

template <typename R>
size_t happly_smem(const HSector &hs, int n_orb) {
    return happly_layout<R>(hs.Db, n_orb, hs.n_alpha, hs.ag).total;
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
                          const DevHam<R> &H, const HSector &hs, double *Epart, int flags) {
    (void)LH;
    dim3 grid(hs.Da * hs.ncb, cfg.B);
    const int threads = happly_threads(hs);
    const int ept = happly_cols_per_thread(hs);
    const size_t smem = happly_smem<R>(hs, H.n_orb);
    const V2<R> *p = static_cast<const V2<R> *>(psi);
    V2<R> *s = static_cast<V2<R> *>(sig);
    cudaError_t e = cudaSuccess;
    switch (ept <= 1 ? 1 : ept <= 2 ? 2 : ept <= 4 ? 4 : ept <= 8 ? 8 : 0) {
        case 1: e = launch_pdl(happly_kernel<R, 1>, grid, dim3(threads), smem, cfg.stream, p, s, cfg.N, H, hs, Epart, flags); break;
        case 2: e = launch_pdl(happly_kernel<R, 2>, grid, dim3(threads), smem, cfg.stream, p, s, cfg.N, H, hs, Epart, flags); break;
        case 4: e = launch_pdl(happly_kernel<R, 4>, grid, dim3(threads), smem, cfg.stream, p, s, cfg.N, H, hs, Epart, flags); break;
        case 8: e = launch_pdl(happly_kernel<R, 8>, grid, dim3(threads), smem, cfg.stream, p, s, cfg.N, H, hs, Epart, flags); break;
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_reduce(const LaunchCfg &cfg, const double *Epart, int n_tiles_h,
                          const double *gpart, int tile_stride, const int32_t *op_tiles,
                          int K, const int32_t *k_ptr,
                          const int32_t *k_ops, const double *op_scale, double shift,
                          int rayleigh, double *E, double *grad) {
    if (grad && tile_stride <= kReduceSerialMax) {
        dim3 grid(std::max(1, (K + kThreads - 1) / kThreads), cfg.B);
        const cudaError_t e = launch_pdl(reduce_serial_kernel, grid, dim3(kThreads), 0, cfg.stream, Epart,
                                         n_tiles_h, gpart, tile_stride, op_tiles, cfg.n_ops, K, k_ptr,
                                         k_ops, op_scale, shift, rayleigh, E, grad);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
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
    UCCSD_SET((happly_kernel<float, 1>));
    UCCSD_SET((happly_kernel<float, 2>));
    UCCSD_SET((happly_kernel<float, 4>));
    UCCSD_SET((happly_kernel<float, 8>));
    UCCSD_SET((happly_kernel<double, 1>));
    UCCSD_SET((happly_kernel<double, 2>));
    UCCSD_SET((happly_kernel<double, 4>));
    UCCSD_SET((happly_kernel<double, 8>));
#undef UCCSD_SET
    return cudaSuccess;
}

#define UCCSD_INST(R)                                                                          \
    template size_t happly_smem<R>(const HSector &, int);                                      \
    template cudaError_t launch_cs<R>(const LaunchCfg &, const double *, int, const int32_t *, \
                                      const double *, void *);                                 \
    template cudaError_t launch_happly<R>(const LaunchCfg &, const void *, void *, int,        \
                                          const DevHam<R> &, const HSector &, double *, int);
UCCSD_INST(float)
UCCSD_INST(double)
#undef UCCSD_INST

}  // namespace uccsd
