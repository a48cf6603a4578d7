// Library context (the opaque uccsd_ctx of include/uccsd.h).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/uccsd.h"
#include "jw.hpp"
#include "kernels.cuh"
#include "plan.hpp"

namespace uccsd {
// Columns (beta strings) per H-apply CTA.
inline constexpr int kHColBlock = 2048;
inline constexpr int kHL = 0;  // unused by the row layout
// Shared memory budget of one compact sweep tile (forward: one vector,
// adjoint: phi and lambda), bytes.
inline constexpr size_t kSweepBudget = 200 * 1024;
}  // namespace uccsd

namespace uccsd {
// Gate status words (gate.cu): a word of a pinned pool allocated once per
// process, and its return.
uint32_t *gate_status_take();
void gate_status_give(uint32_t *w);
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
    // Stream of the set-up transfers (uploads, clears, downloads).  By default
    // the context's own non-blocking stream, waited on by the host after each
    // transfer.  After uccsd_set_setup_stream with a caller stream the
    // transfers are enqueued there from pinned staging and nothing waits: the
    // caller orders later work after that stream.
    cudaStream_t setup = nullptr;
    cudaStream_t own_setup = nullptr;
    // evaluation stream of uccsd_energy_grad_batched (forked from and joined
    // back into the caller's stream) and its fork / join events
    cudaStream_t aux = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool setup_async = false;
    char *stage = nullptr;  // pinned staging of asynchronous uploads
    size_t stage_cap = 0, stage_off = 0;
    cudaEvent_t stage_ev = nullptr;  // recorded on `setup` after the last staged copy

    // problem
    int n_orb = 0, n = 0;
    bool have_h = false, have_ref = false, have_exc = false;
    int n_alpha = 0, n_beta = 0;
    uint32_t hf = 0;       // reference determinant (qubit bits)
    int layout = 0;        // 0 full 2^n vector, 1 electron-sector array (UCCSD_LAYOUT_*)
    uint32_t hf_addr = 0;  // address of the reference amplitude in a slot
    // electron-sector addressing (rank(sa) * Db, rank(sb)) in any layout, and
    // whether the forward's runs pass the state, and the adjoint's runs phi
    // and lambda, on in that compact order
    const uint32_t *sec_aoff = nullptr, *sec_boff = nullptr;
    bool adj_compact = false, fwd_compact = false;
    uccsd::CompiledH H;
    std::vector<int32_t> spec_s1a, spec_s1b;  // spectator row of each alpha / beta pair group
    int K = 0, order = 1, M = 1;
    std::vector<int32_t> ijab, op_k;
    std::vector<double> op_scale;
    uccsd::SweepPlan fwd, adj;
    uccsd::SweepArgs fwd_args, adj_args;
    // entry maps of the forward and adjoint plans (null when too large):
    // set as SweepArgs / SweepOut::emap where a run reads or writes vectors
    // in the sector order
    const uint32_t *fwd_emap = nullptr, *adj_emap = nullptr;
    // Pair lists of the forward and adjoint plans: device copies shared with
    // every context of the same plan (not counted in `bytes`), and their hashes
    std::shared_ptr<void> lists_held[2];
    uint64_t list_key[2] = {0, 0};
    // shape of the last complete set_excitations (plans, tables and slots
    // depend on it and the list only, not on the integrals)
    bool exc_valid = false;
    int exc_n = 0, exc_na = 0, exc_nb = 0, exc_layout = -1;
    std::vector<uccsd::CompiledExc> exc;  // list order
    // Trotter-free ansatz: plan with every excitation once (built on first use)
    uccsd::SweepPlan tf;
    uccsd::SweepArgs tf_args;
    bool tf_ready = false;
    int LH = uccsd::kHL;
    int B = 1;          // reserved slots
    bool state_valid = false;

    // device memory: name -> (ptr, bytes)
    std::map<std::string, std::pair<void *, size_t>> mem;

    // Hamiltonian views
    uccsd::DevHam<float> hf32;
    uccsd::DevHam<double> hf64;
    uccsd::HSector hsec;
    uccsd::HSector hsec_full;  // hsec with full-layout addressing (caller states)
    uccsd::HSector hsec_sec;   // hsec with the compact sector addressing (any layout)
    uint32_t hf_sec = 0;       // address of the reference amplitude in the compact order
    // combinatorial rank tables (shared by the sweeps and the H-apply)
    const uint16_t *comb_combos = nullptr, *comb_ranks = nullptr;
    const int32_t *comb_offs = nullptr;
    std::vector<int32_t> comb_offs_host;

    // diagonal in fixed point; energy shift (the reference determinant's
    // diagonal energy) applied to H on the device and added back in FP64
    std::vector<long long> diag_qa, diag_qb;
    double diag_unit = 0.0;
    double shift = 0.0;

    // device optimiser (fixed-step L-BFGS)
    int opt_m = 0, opt_steps = 0;
    double opt_max_step = 0.0, opt_first = 0.0;
    // its record (4 meta ints, then the energy history) in the process's
    // mapped pinned pool (capi.cpp), or null: device buffers opt_meta and
    // opt_hist; opt_rec_dev is the record's device address
    double *opt_rec = nullptr, *opt_rec_dev = nullptr;

    // gate of the serving loop (uccsd_gate_enqueue): its status word in
    // mapped pinned memory (1 released, 2 gave up), the event after the gate
    uint32_t *gate_status = nullptr;  // a word of the process's pool (gate.cu)
    cudaEvent_t gate_ev = nullptr;
    cudaEvent_t mark_ev = nullptr;  // uccsd_stream_mark
    bool marked = false;
    bool gate_pending = false;

    // captured evaluation graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_kernels = 0;

    // profiling
    bool profiling = false;
    uccsd_profile_t prof{};
    std::vector<cudaEvent_t> events;
};
