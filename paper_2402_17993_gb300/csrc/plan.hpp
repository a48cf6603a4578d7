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
    std::vector<RunDev> runs;
    std::vector<OpDev> ops;   // ops of run r at [runs[r].op_begin, runs[r].op_end)
    int L = 0;                // tile bits
};

// Split the schedule into maximal consecutive runs whose flips fit in L tile
// bits that always contain the low bits 0..c_min-1.  Each run's tile is the
// union of its flips padded with the lowest unused bits.
SweepPlan plan_sweep(int n_qubits, int L, int c_min, const std::vector<CompiledExc> &exc,
                     const std::vector<int32_t> &op_k);

}  // namespace uccsd
