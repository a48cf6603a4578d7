// Launch wrappers of the UCCSD CUDA kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "common.hpp"

namespace uccsd {

// Device copy of the compiled Hamiltonian for one precision R.
template <typename R>
struct DevHam {
    const GroupT<R> *groups = nullptr;  // sorted by segment, diagonal segment last
    const int32_t *seg_begin = nullptr; // n_seg + 1
    const uint32_t *seg_d = nullptr;    // high-part XOR of each segment
    int n_seg = 0;
    const R *spec = nullptr;            // spectator rows [row][4]
    // Diagonal group as an occupation quadratic form in 64-bit fixed point
    // (one unit = diag_unit Ha), summed exactly:
    //   d(x) - shift = q0 + sum_{q in occ(x)} qa[q] + sum_{q<r in occ(x)} qb[q*n + r]
    const long long *diag_qa = nullptr; // n
    const long long *diag_qb = nullptr; // n*n (q < r)
    long long diag_q0 = 0;
    double diag_unit = 0.0;
    int has_diag = 0;
    int n = 0;                          // qubits (row length of diag_qb)
};

// Compact sector tiles of the H-apply: a tile is the set of sector
// amplitudes with fixed values of the bits above the low LH bits; its entries
// form a [C(LH/2, a)] x [C(LH/2, b)] array indexed by the ranks of the low
// alpha and beta bit strings among strings of equal popcount.
struct HSector {
    const uint16_t *combos = nullptr;    // strings sorted by (popcount, value), per bit count
    const uint16_t *ranks = nullptr;     // rank of a string within its popcount class
    const int32_t *comb_offs = nullptr;  // class offsets, 17 per bit count
    const uint32_t *spread = nullptr;    // 2^(LH/2) alpha then 2^(LH/2) beta string deposits
    int n_alpha = 0, n_beta = 0;
    int max_entries = 0;                 // largest compact tile
};

struct LaunchCfg {
    int n = 0;           // qubits
    size_t N = 0;        // 2^n
    int B = 1;           // slots in this call
    int n_ops = 0;
    cudaStream_t stream = nullptr;
};

// cs[b][o] = (cos, sin)(theta[b][op_k[o]] * op_scale[o]) computed in FP64,
// stored in R.
template <typename R>
cudaError_t launch_cs(const LaunchCfg &cfg, const double *theta, int K, const int32_t *op_k,
                      const double *op_scale, void *cs);

// Tables shared by the compact-tile sweeps (see plan.hpp).
struct SweepArgs {
    const uint16_t *combos = nullptr;    // strings sorted by (popcount, value), per bit count
    const uint16_t *ranks = nullptr;     // rank of a string within its popcount class
    const int32_t *comb_offs = nullptr;  // class offsets, 17 per bit count
    const uint32_t *spread = nullptr;    // per run: tile string -> global bits
    uint32_t amask = 0;                  // alpha qubits (even positions)
    int n_alpha = 0, n_beta = 0;
};

template <typename R>
cudaError_t launch_forward_sweep(const LaunchCfg &cfg, void *psi, const CRunDev &run,
                                 const COpDev *ops, const void *cs, const SweepArgs &sa,
                                 int init_hf, uint32_t hf);

template <typename R>
cudaError_t launch_adjoint_sweep(const LaunchCfg &cfg, void *phi, void *lam, const CRunDev &run,
                                 const COpDev *ops, const void *cs, const SweepArgs &sa,
                                 double *gpart, int tile_stride);

// |HF> in every slot (used when the schedule is empty).
template <typename R>
cudaError_t launch_set_hf(const LaunchCfg &cfg, void *psi, uint32_t hf);

// Dynamic shared memory opt-in of the sweep kernels.
cudaError_t configure_sweep_kernels(size_t max_smem);

template <typename R>
cudaError_t launch_happly(const LaunchCfg &cfg, const void *psi, void *sig, int LH,
                          const DevHam<R> &H, const HSector &hs, double *Epart, int store_sigma);

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

// Shared memory of the H-apply kernel for its largest compact tile.
template <typename R>
size_t happly_smem(int max_entries);

// One-time kernel attribute set-up (dynamic shared memory opt-in).
cudaError_t configure_kernels();

}  // namespace uccsd
