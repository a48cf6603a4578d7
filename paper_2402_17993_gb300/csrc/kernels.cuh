// Launch wrappers of the UCCSD CUDA kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "common.hpp"

namespace uccsd {

// Device copy of the compiled Hamiltonian for one precision R, by group class.
template <typename R>
struct DevHam {
    const MixT<R> *mix = nullptr;  // [n_pairs * n_pairs], alpha pair major
    const MixO<R> *mixo = nullptr; // [n_orb^4], ordered alpha and beta excitations
    // same-spin doubles by ordered target pattern: entry ((o1 n + o2) n + v1) n + v2
    // (o1 < o2 occupied and v1 < v2 empty in the target) holds the LUT value of
    // the source occupying v1, v2 and the group's Jordan-Wigner mask
    const MixO<R> *d2ao = nullptr;
    const MixO<R> *d2bo = nullptr;
    // beta doubles by pair index: entry pair(o1, o2) * n_pairs + pair(v1, v2)
    // (o1 < o2 occupied, v1 < v2 empty in the target), the value times the
    // excitation's own part of the Jordan-Wigner sign
    const R *d2bs = nullptr;
    const SglT<R> *s1a = nullptr;  // [n_pairs] alpha singles
    const SglT<R> *s1b = nullptr;  // [n_pairs] beta singles
    const DblT<R> *d2a = nullptr;  // [n_quads] alpha doubles
    const DblT<R> *d2b = nullptr;  // [n_quads] beta doubles
    const R *spec = nullptr;       // spectator rows [row][4]
    // Beta-spectator sums per column (Db columns, the reference's beta
    // strings), zero for groups without spectator rows:
    //   bspec_a[(pa * 2 + sel) * Db + c]: alpha pair group pa, source side sel,
    //     summed over the occupied beta orbitals of column c;
    //   bspec_b[t * Db + c]: the t-th beta single of column c (order of
    //     HSector::bsing), summed over the source's occupied beta orbitals
    //     other than the created one.
    const R *bspec_a = nullptr;
    const R *bspec_b = nullptr;
    // Diagonal group as an occupation quadratic form in 64-bit fixed point
    // (one unit = diag_unit Ha), summed exactly:
    //   d(x) - shift = q0 + sum_{q in occ(x)} qa[q] + sum_{q<r in occ(x)} qb[q*n + r]
    const long long *diag_qa = nullptr; // n
    const long long *diag_qb = nullptr; // n*n (q < r)
    // The part of that form over the beta qubits of each column (Db
    // entries, the reference's beta strings); the H-apply adds the alpha
    // part and the alpha-beta pairs per row.
    const long long *diag_col = nullptr;
    long long diag_q0 = 0;
    double diag_unit = 0.0;
    int has_diag = 0;
    int n = 0;                          // qubits
    int n_orb = 0, n_pairs = 0;
};

// Sector layout of the H-apply: a row is one alpha string of the sector
// (n_alpha electrons), its columns are the beta strings (n_beta electrons),
// both in rank order (rank = position among strings of equal popcount).
// A CTA owns the columns [cb * colblock, (cb + 1) * colblock) of one row.
struct HSector {
    const uint16_t *astr = nullptr;    // Da alpha strings
    const uint16_t *bstr = nullptr;    // Db beta strings
    const uint16_t *brank = nullptr;   // rank of any n_orb-bit string in its popcount class
    const uint32_t *aspread = nullptr; // alpha string -> qubit bits (2^n_orb)
    const uint32_t *bspread = nullptr; // beta string -> qubit bits (2^n_orb)
    // State addressing: the amplitude of determinant (alpha string sa, beta
    // string sb) of a slot is at aoff[sa] + boff[sb].  Full 2^n layout: the
    // qubit bits (aoff = aspread, boff = bspread); sector layout: rank(sa) * Db
    // and rank(sb).
    const uint32_t *aoff = nullptr;
    const uint32_t *boff = nullptr;
    const int32_t *binom = nullptr;    // binom[t * 5 + k], t < 16, k <= 4
    // Beta single excitations of every column, [s][Db] with s over the
    // column's occupied j (ascending) then virtual b (ascending):
    // x = rank of the source string yb = bstr ^ {j, b} | (j * n_orb + b) << 16,
    // y = c | (2 * pair_index(min(j, b), max(j, b)) + (b > j)) << 16 with c
    // the column's part of the Jordan-Wigner sign: the parity of the
    // column's occupied orbitals below j, plus those below b, plus (b > j).
    // n_bs = n_beta * (n_orb - n_beta) per column.
    const uint2 *bsing = nullptr;
    // The same excitations for the mixed groups, [s][Db]: rank of the source
    // string | (j * n_orb + b + n_orb^2 * pi) << 16, pi the parity of the
    // column's occupied beta orbitals strictly between j and b (selects the
    // negated half of the H-apply's staged mixed table).
    const uint32_t *bmix = nullptr;
    int n_bs = 0;
    int ag = 1;  // alpha singles staged per phase of the H-apply (1..4)
    int n_alpha = 0, n_beta = 0;
    int Da = 0, Db = 0;
    int colblock = 0, ncb = 1;
};

struct LaunchCfg {
    int n = 0;           // qubits
    size_t N = 0;        // amplitudes per slot: 2^n (full layout) or Da * Db (sector layout)
    int B = 1;           // slots in this call
    int n_ops = 0;
    cudaStream_t stream = nullptr;
};

// cs[b][o] = (cos, sin)(a) with a = theta[b][op_k[o]] * op_scale[o],
// computed in FP64 and stored in R; the FP32 state stores (1 - cos, sin)(a)
// (its rotation form, see sweep.cu).
template <typename R>
cudaError_t launch_cs(const LaunchCfg &cfg, const double *theta, int K, const int32_t *op_k,
                      const double *op_scale, void *cs);

// Tables shared by the compact-tile sweeps (see plan.hpp).
struct SweepArgs {
    const uint16_t *combos = nullptr;    // strings sorted by (popcount, value), per bit count
    const uint16_t *ranks = nullptr;     // rank of a string within its popcount class
    const int32_t *comb_offs = nullptr;  // class offsets, 17 per bit count
    const uint32_t *spread = nullptr;    // per run: tile string -> orbital string
    const uint32_t *aoff = nullptr;      // state addressing (see HSector)
    const uint32_t *boff = nullptr;
    // precomputed pair lists (PairLists of plan.hpp), null when the plan has none
    const int2 *op_pl = nullptr;
    const uint2 *pairs = nullptr;
    uint32_t amask = 0;                  // alpha qubits (even positions)
    int n_alpha = 0, n_beta = 0;
    // the plan's entry maps (sector index of each tile entry, from
    // CRunDev::emap_base) when the vectors read are in the sector order
    // (aoff / boff the sector addressing), else null: the tables above
    const uint32_t *emap = nullptr;
};

// Where a sweep run leaves its vectors after its factors (the forward: the
// state in phi; the adjoint: phi and lambda): slot b of each at phi + b * N
// (same for lam), amplitude of determinant (alpha string sa, beta string sb)
// at aoff[sa] + boff[sb].  phi == nullptr (adjoint only): nowhere, after the
// last run of the sweep, since nothing reads the vectors afterwards.
struct SweepOut {
    void *phi = nullptr, *lam = nullptr;
    size_t N = 0;
    const uint32_t *aoff = nullptr, *boff = nullptr;
    const uint32_t *emap = nullptr;  // as SweepArgs::emap, for the vectors written
};

// psi, cfg.N and sa.aoff / sa.boff address the state the run reads (unused
// when init_hf is set: the run starts from the reference determinant).
template <typename R>
cudaError_t launch_forward_sweep(const LaunchCfg &cfg, void *psi, const CRunDev &run,
                                 const COpDev *ops, const void *cs, const SweepArgs &sa,
                                 int init_hf, uint32_t hf, const SweepOut &out);

// phi, lam, cfg.N and sa.aoff / sa.boff address the vectors the run reads.
template <typename R>
cudaError_t launch_adjoint_sweep(const LaunchCfg &cfg, void *phi, void *lam, const CRunDev &run,
                                 const COpDev *ops, const void *cs, const SweepArgs &sa,
                                 double *gpart, int tile_stride, const SweepOut &out);

// |HF> in every slot (used when the schedule is empty).
template <typename R>
cudaError_t launch_set_hf(const LaunchCfg &cfg, void *psi, uint32_t hf);

// Trotter-free ansatz (Eq. 3): w (+)= scale * sum_k coef[k] G_k u over one
// run of a plan holding each excitation once (first_run: w starts at zero).
template <typename R>
cudaError_t launch_gen_apply(const LaunchCfg &cfg, const void *u, void *w, const CRunDev &run,
                             const COpDev *ops, const double *coef, double scale,
                             const SweepArgs &sa, int first_run);
// acc = u = |HF> on the electron sector (slot 0).
template <typename R>
cudaError_t launch_sector_init(const LaunchCfg &cfg, void *acc, void *u, const HSector &hs,
                               uint32_t hf);
// acc += w on the electron sector; u_out (may be null) = the new acc.
template <typename R>
cudaError_t launch_sector_axpy(const LaunchCfg &cfg, void *acc, const void *w, void *u_out,
                               const HSector &hs);

// Trotter-free gradient integrand: gpart[k][t] = tile-t partial of
// Re <lam|G_k|phi> for the factors of one run (plan holding each excitation once).
template <typename R>
cudaError_t launch_gen_dot(const LaunchCfg &cfg, const void *phi, const void *lam,
                           const CRunDev &run, const COpDev *ops, const SweepArgs &sa,
                           double *gpart, int tile_stride);
// g[k] = (init ? 0 : g[k]) + 2 weight sum_t gpart[k][t], t < op_tiles[k].
cudaError_t launch_tf_grad_accum(const LaunchCfg &cfg, const double *gpart, int tile_stride,
                                 const int32_t *op_tiles, int K, double weight, double *g,
                                 int init);
// dst = src on the electron sector.
template <typename R>
cudaError_t launch_sector_copy(const LaunchCfg &cfg, void *dst, const void *src, const HSector &hs);

// Gradient partial slots per tile that the adjoint launch of `run` writes:
// one per warp for the pair-list kernels, one for the builder kernels.
int adjoint_partials_per_tile(const CRunDev &run, bool lists);

// Dynamic shared memory opt-in of the sweep kernels.
cudaError_t configure_sweep_kernels(size_t max_smem);

// H-apply flags: store sigma (energy-only calls skip it); the FP32 slots
// hold complex (re, im) amplitudes (a caller's state) instead of the real
// hi + lo amplitudes of the library's FP32 state (see amp.cuh).
constexpr int kHApplyStoreSigma = 1;
constexpr int kHApplyComplex32 = 2;
template <typename R>
cudaError_t launch_happly(const LaunchCfg &cfg, const void *psi, void *sig, int LH,
                          const DevHam<R> &H, const HSector &hs, double *Epart, int flags);

// E[b] from the per-tile partials (e', n) of sum Re(conj psi (H - shift) psi)
// and sum |psi|^2: E = shift * n + e' (rayleigh = 0) or shift + e'/n
// (rayleigh = 1); the gradient is divided by n when rayleigh = 1.
// gpart[b][o][t] holds op_tiles[o] tile partials of factor o (row stride
// tile_stride).
cudaError_t launch_reduce(const LaunchCfg &cfg, const double *Epart, int n_tiles_h,
                          const double *gpart, int tile_stride, const int32_t *op_tiles,
                          int K, const int32_t *k_ptr,
                          const int32_t *k_ops, const double *op_scale, double shift,
                          int rayleigh, double *E, double *grad);

// Shared memory of the H-apply kernel.
template <typename R>
size_t happly_smem(const HSector &hs, int n_orb);

// Threads of an H-apply CTA (a column block, one or more columns per
// thread) and the columns each thread takes.  At one column per thread the
// FP32 kernel stages the alpha singles' source rows in 16-byte chunks and
// reads the mixed groups' beta singles in the order of happly_mixed_order.
constexpr int kRowThreads = 256;
inline int happly_threads(const HSector &hs) {
    const int t = ((hs.colblock + 31) / 32) * 32;
    return t < 32 ? 32 : t > kRowThreads ? kRowThreads : t;
}
inline int happly_cols_per_thread(const HSector &hs) {
    const int t = happly_threads(hs);
    return (hs.colblock + t - 1) / t;
}

// Fixed-step L-BFGS update of theta (K doubles, device) from the gradient g
// and energy E of the evaluation at theta; state holds 2 m K + m + 3 K
// doubles, meta 4 ints (zeroed to start); E is recorded in E_hist[step].
cudaError_t launch_lbfgs(cudaStream_t stream, int K, int m, double max_step, double first_scale,
                         double *theta, const double *E, const double *g, double *state,
                         int *meta, double *E_hist, int max_steps);

// One-time kernel attribute set-up (dynamic shared memory opt-in).
cudaError_t configure_kernels();

}  // namespace uccsd
