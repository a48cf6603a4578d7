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

// Shared-memory tile of a run: the largest compact tile rounded up to 16
// entries, then 32 zeroed scratch entries that the padding pairs of the
// precomputed lists rotate (no effect: they stay zero).
constexpr int kTileScratch = 32;
#ifdef __CUDACC__
#define UCCSD_HD __host__ __device__
#else
#define UCCSD_HD
#endif
UCCSD_HD inline int tile_scratch(int max_entries) { return (max_entries + 15) & ~15; }
UCCSD_HD inline int tile_alloc(long long max_entries) { return tile_scratch(int(max_entries)) + kTileScratch; }

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
// descriptors, cos/sin values (one amplitude each) and pair-list entries
// (8 bytes each) and (lmax <= kStageLmax) the staged tables.
size_t sweep_smem_bytes(long long entries, long long da, long long db, size_t amp_bytes,
                        int nvec, int n_ops_run, int lmax);

// Split the schedule into maximal consecutive runs whose flipped bits fit in
// a tile bit set whose largest compact tile of `nvec` vectors of
// `amp_bytes` amplitudes stays within `budget` bytes.
SweepPlan plan_sweep(int n_qubits, int n_alpha, int n_beta, size_t amp_bytes, int nvec,
                     size_t budget, const std::vector<CompiledExc> &exc,
                     const std::vector<int32_t> &op_k);

// Precomputed pair lists of a sweep plan.  For every run, every electron
// count class (a, b) of its tiles (class index a * (Lb + 1) + b) and every
// factor of the run, the factor's pairs in tile-entry coordinates: pair word
// 2i = the occupied-side entry e, word 2i + 1 = the partner entry e', except
// that a pair whose strings have odd Jordan-Wigner parity is stored as
// (e', e): rotating that order with the even-parity sign is the same
// rotation, so no per-pair sign is stored.  The pairs of (run r, class c,
// factor o) start at
// pair op_pl[2 * (runs[r].pl_base + c * n_ops_r + o)] and number
// op_pl[2 * (...) + 1].  Within a factor the pairs come in aligned groups of
// bank_group pairs (the lanes of one shared-memory wavefront: 16 for 8-byte,
// 8 for 16-byte amplitudes) whose e and e' are distinct modulo bank_group,
// so no group has a bank conflict; groups are completed with padding pairs
// on the tile's scratch entries (tile_scratch(max_entries) + r), which hold
// zeros, so the counts include the padding.
struct PairLists {
    std::vector<uint32_t> pairs;
    std::vector<int32_t> op_pl;
    size_t n_pairs = 0;
};

// Fill `out` and set runs[r].pl_base for every run; false (plan untouched,
// pl_base = -1) when the lists would hold more than max_pairs pairs.
bool build_pair_lists(int n_qubits, int n_alpha, int n_beta, size_t max_pairs, SweepPlan *plan,
                      PairLists *out, int bank_group);

// One pair of a plan's lists in determinant space: the sweep loads the
// amplitudes of `first` and `second` and rotates
//   first' = c first - sign s second,  second' = c second + sign s first
// (c, s the factor's cos and sin).  Padding pairs have first = second =
// 0xFFFFFFFF.  e, e2: tile entries; index: position in the factor's list.
struct ExpandedPair {
    int32_t factor;
    uint32_t first, second;
    int32_t sign;
    int32_t e, e2, index;
};
// Every pair of every run, tile and factor of `plan` with lists L (host
// check of the lists against an independent generator action).
std::vector<ExpandedPair> expand_pair_lists(int n_qubits, int n_alpha, int n_beta,
                                            const SweepPlan &plan, const PairLists &L);

// Entry maps of a plan: the sector index (alpha string rank x C(n_orb,
// n_beta) + beta string rank, strings ranked in ascending order within
// their popcount) of every entry e = ia * Db + ib of every tile of every run,
// as the sweep kernels' tile view orders them; run r's tiles at max_entries
// entries each from runs[r].emap_base (set here).  Unused slots are 0.
std::vector<uint32_t> build_entry_map(int n_qubits, int n_alpha, int n_beta, SweepPlan *plan);
// The determinants of tile `tile` of run r in entry order, decoded by
// depositing the tile strings into the tile's qubit positions (a check of
// the maps by another route); empty for a tile without sector entries.
std::vector<uint32_t> tile_entry_dets(int n_qubits, int n_alpha, int n_beta, const CRunDev &r,
                                      int tile);

// Order of every column's beta single excitations in the FP32 H-apply's
// mixed groups (one column per thread, staged source rows in 16-byte
// chunks).  Column c's k-th single j -> b in natural order (j occupied
// ascending, then b empty ascending) is taken at slot t when
// order[t * Db + c] == k; Db = C(n_orb, n_beta) columns in ascending string
// order.  Per aligned group of eight columns (the lanes of one wavefront of
// 16-byte shared-memory loads) the slots are chosen to minimise the bank
// conflicts of the loads of the staged mixed table and source rows; any
// order gives the same contributions, summed in that order.
std::vector<uint8_t> happly_mixed_order(int n_orb, int n_beta);

// Combinatorial tables for bit strings of m <= kCombMax bits: for each m,
// the 2^m strings sorted by (popcount, value) at combos[2^m - 1 ...], the
// rank of each string among those of equal popcount at rank[2^m - 1 + s],
// and offs[m * 17 + c] = start of popcount class c (c = 0..m+1).
constexpr int kCombMax = 15;
void build_comb_tables(std::vector<uint16_t> *combos, std::vector<uint16_t> *rank,
                       std::vector<int32_t> *offs);

}  // namespace uccsd
