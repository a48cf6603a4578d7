// Host-side excitation list (Eq. 4), Trotter schedule (Eq. 5/6) and the
// shared-memory run planner of the excitation sweeps.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "common.hpp"
#include "jw.hpp"

namespace uccsd {

// Reference determinant bits: n_alpha lowest even and n_beta lowest odd qubits.
uint64_t hf_bits(int n_alpha, int n_beta);

// Spin-conserving singles then doubles, lexicographic (Eq. 4).
std::vector<int32_t> build_uccsd_list(int n_orb, int n_alpha, int n_beta);

// Schedule of Eq. 5 (order 1) or Eq. 6 (order 2): factor o applies
// exp(theta[op_k[o]] * op_scale[o] * G).
void build_schedule(int K, int order, int M, std::vector<int32_t> *op_k,
                    std::vector<double> *op_scale);

struct SweepPlan {
    std::vector<CRunDev> runs;
    std::vector<COpDev> ops;       // ops of run r at [runs[r].op_begin, runs[r].op_end)
    std::vector<uint32_t> spread;  // per run: tile alpha / beta string -> orbital string
    std::vector<int32_t> op_tiles; // per schedule factor: tiles of its run
    int max_tiles = 1;
    int max_entries = 1;
};

// Largest compact tile (entries) of a tile bit set: the sector leaves
// a alpha electrons for the tile's La alpha bits for every feasible split.
long long max_tile_entries(int n_qubits, int n_alpha, int n_beta, uint32_t tmask);
// Largest alpha / beta string counts C(La, a), C(Lb, b) of a tile bit set.
void max_tile_sides(int n_qubits, int n_alpha, int n_beta, uint32_t tmask, long long *da,
                    long long *db);
// Bit counts up to which a sweep CTA stages the combinatorial tables in
// shared memory.
constexpr int kStageLmax = 10;
// Shared memory of the staged combinatorial tables for bit counts <= lmax.
size_t sweep_table_bytes(int lmax);
// Shared memory of one sweep CTA: nvec tiles, the two double-buffered
// alpha/beta pair-side lists (8 bytes per string), the run's factor
// descriptors and cos/sin values (one amplitude each) and (lmax <=
// kStageLmax) the staged tables.
size_t sweep_smem_bytes(long long entries, long long da, long long db, size_t amp_bytes,
                        int nvec, int n_ops_run, int lmax);

// Split the schedule into maximal consecutive runs whose flipped bits fit in
// a tile bit set whose largest compact tile of `nvec` vectors of
// `amp_bytes` amplitudes stays within `budget` bytes.
SweepPlan plan_sweep(int n_qubits, int n_alpha, int n_beta, size_t amp_bytes, int nvec,
                     size_t budget, const std::vector<CompiledExc> &exc,
                     const std::vector<int32_t> &op_k);

// Combinatorial tables for bit strings of m <= kCombMax bits: for each m,
// the 2^m strings sorted by (popcount, value) at combos[2^m - 1 ...], the
// rank of each string among those of equal popcount at rank[2^m - 1 + s],
// and offs[m * 17 + c] = start of popcount class c (c = 0..m+1).
constexpr int kCombMax = 15;
void build_comb_tables(std::vector<uint16_t> *combos, std::vector<uint16_t> *rank,
                       std::vector<int32_t> *offs);

}  // namespace uccsd
