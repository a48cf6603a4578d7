// Library context (the opaque uccsd_ctx of include/uccsd.h).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/uccsd.h"
#include "jw.hpp"
#include "kernels.cuh"
#include "plan.hpp"

namespace uccsd {
// Tile bits of the kernels per precision (shared memory per CTA):
//   forward  FP32 13 (64 KiB), FP64 12 (64 KiB)
//   adjoint  FP32 12 (2 x 32 KiB), FP64 11 (2 x 32 KiB)
//   H-apply  12 (32 / 64 KiB)
inline constexpr int kFwdL[2] = {12, 13};
inline constexpr int kAdjL[2] = {11, 12};
inline constexpr int kHL = 12;
inline constexpr int kCmin = 3;
}  // namespace uccsd

struct uccsd_ctx {
    int device = 0;
    int prec = 0;  // 0 FP64, 1 FP32 state
    size_t budget = 0;
    size_t bytes = 0;
    std::string err;
    bool failed = false;
    uint64_t launches = 0;
    cudaStream_t last_stream = nullptr;

    // problem
    int n_orb = 0, n = 0;
    bool have_h = false, have_ref = false, have_exc = false;
    int n_alpha = 0, n_beta = 0;
    uint32_t hf = 0;
    uccsd::CompiledH H;
    int K = 0, order = 1, M = 1;
    std::vector<int32_t> ijab, op_k;
    std::vector<double> op_scale;
    uccsd::SweepPlan fwd, adj;
    int LH = uccsd::kHL;
    int B = 1;          // reserved slots
    bool state_valid = false;

    // device memory: name -> (ptr, bytes)
    std::map<std::string, std::pair<void *, size_t>> mem;

    // Hamiltonian views
    uccsd::DevHam<float> hf32;
    uccsd::DevHam<double> hf64;
    uccsd::HSector hsec;

    // diagonal in fixed point; energy shift (the reference determinant's
    // diagonal energy) applied to H on the device and added back in FP64
    std::vector<long long> diag_qa, diag_qb;
    double diag_unit = 0.0;
    double shift = 0.0;

    // profiling
    bool profiling = false;
    uccsd_profile_t prof{};
    std::vector<cudaEvent_t> events;
};
