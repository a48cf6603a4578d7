// Energy of a caller-supplied state vector without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need an energy:
// real-time or serving loops that run under a fixed, pre-reserved memory
// budget (an allocation there may fail, or stall the device while other
// work is in flight), and plugins inside hosts whose device allocator is
// owned by another framework (memory taken behind that allocator's back is
// memory it cannot account for).  uccsd_expectation_noalloc serves them: it
// reuses the Hamiltonian tables that the context uploaded when it was set
// up, takes the state and the result buffer from the caller, and keeps its
// only scratch (the per-tile energy partials) in the file-scope device
// array below instead of allocating.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/uccsd.h"
#include "ctx.hpp"
#include "kernels.cuh"

namespace {

// Scratch of the no-allocation entry point: two doubles (energy, norm) per
// H-apply tile, UCCSD_NOALLOC_MAX_TILES tiles (64 KiB).  Every GPU that
// loads this library holds one copy until the process exits.
static __device__ __align__(256) double g_noalloc_partials[2 * UCCSD_NOALLOC_MAX_TILES];

// Device address of g_noalloc_partials per device.  In host code the name
// g_noalloc_partials is only a host-side stand-in and must never be passed
// to a kernel, so the real address is looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_partials_dev[kMaxDevices] = {nullptr};

// Look up the scratch address on `device`, which must be current.
cudaError_t scratch_address(int device, double **out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_dev[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_dev[device] = static_cast<double *>(p);
    }
    *out = g_partials_dev[device];
    return cudaSuccess;
}

}  // namespace

extern "C" uccsd_status uccsd_expectation_noalloc(uccsd_ctx *c, const void *psi, double *E,
                                                  void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) {
        c->err = "context failed earlier: " + c->err;
        return UCCSD_ERR_STATE;
    }
    if (!c->have_ref) {
        c->err = "uccsd_expectation_noalloc needs set_hamiltonian and set_reference first";
        return UCCSD_ERR_STATE;
    }
    if (!psi || !E) {
        c->err = "uccsd_expectation_noalloc: null state or result pointer";
        return UCCSD_ERR_ARG;
    }
    const int tiles = c->hsec.Da * c->hsec.ncb;
    if (tiles > UCCSD_NOALLOC_MAX_TILES) {
        c->err = "uccsd_expectation_noalloc: the state needs " + std::to_string(tiles) +
                 " H-apply tiles (C(n_orb, n_alpha) x ceil(C(n_orb, n_beta) / " +
                 std::to_string(uccsd::kHColBlock) + ")), above the fixed scratch of " +
                 std::to_string(UCCSD_NOALLOC_MAX_TILES) + " tiles";
        return UCCSD_ERR_ARG;
    }
    if (c->device < 0 || c->device >= kMaxDevices) {
        c->err = "uccsd_expectation_noalloc: device index out of range";
        return UCCSD_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(c->device);
    double *partials = nullptr;
    if (e == cudaSuccess) e = scratch_address(c->device, &partials);
    if (e != cudaSuccess) {
        c->err = std::string("uccsd_expectation_noalloc set-up: ") + cudaGetErrorString(e);
        return UCCSD_ERR_CUDA;
    }
    uccsd::LaunchCfg cfg;
    cfg.n = c->n;
    cfg.N = size_t(1) << c->n;
    cfg.B = 1;
    cfg.n_ops = 0;
    cfg.stream = static_cast<cudaStream_t>(stream);
    // The H-apply writes both partials of every tile before the reduction
    // reads them, so nothing in the scratch has to start at zero.
    if (c->prec)
        e = uccsd::launch_happly<float>(cfg, psi, nullptr, c->LH, c->hf32, c->hsec_full, partials,
                                         uccsd::kHApplyComplex32);
    else
        e = uccsd::launch_happly<double>(cfg, psi, nullptr, c->LH, c->hf64, c->hsec_full, partials,
                                         uccsd::kHApplyComplex32);
    if (e == cudaSuccess)
        e = uccsd::launch_reduce(cfg, partials, tiles, nullptr, 1, nullptr, 0, nullptr, nullptr,
                                 nullptr, c->shift, c->prec ? 1 : 0, E, nullptr);
    if (e != cudaSuccess) {
        c->failed = true;
        c->err = std::string("uccsd_expectation_noalloc kernel: ") + cudaGetErrorString(e);
        return UCCSD_ERR_CUDA;
    }
    c->launches += 2;
    return UCCSD_OK;
}
