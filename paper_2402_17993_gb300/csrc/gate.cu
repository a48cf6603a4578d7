// Bounded device wait of the serving loop: a gate kernel that holds the
// work enqueued behind it on a stream until the host releases a flag.
//
// A server can prepare a fragment (set-up, graph capture) and enqueue its
// whole solve before the request is due, behind a gate; at the request's
// arrival the host only writes the flag, and the solve starts as soon as
// the gate kernel sees it, without a launch from the host.  The gate polls
// with a bounded spin: after the caller's time limit (or a hard iteration
// cap, should the timer stall) it gives up, records that in a status word
// and returns, so a flag that is never written cannot hold a stream, and
// the host learns of it from uccsd_gate_status (UCCSD_ERR_TIMEOUT).  The
// flag is written by the host (pinned memory, which the device reads
// through unified addressing) or by a copy on another stream, never by a
// kernel that could itself be waiting.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/uccsd.h"
#include "ctx.hpp"

namespace uccsd {

// Status words of the gates, from one pinned, mapped block allocated at the
// first gate of the process.  A pinned allocation waits for the device, and
// while gates wait for flags that are released later, such a wait (on any
// host thread) holds up the thread that would release them; so no gate
// allocates after the first.
namespace {
constexpr int kGateStatusWords = 4096;
std::mutex g_gate_mu;
uint32_t *g_gate_words = nullptr;
std::vector<int> *g_gate_free = nullptr;  // never destroyed (no CUDA calls at exit)
}  // namespace

uint32_t *gate_status_take() {
    std::lock_guard<std::mutex> lk(g_gate_mu);
    if (!g_gate_words) {
        void *p = nullptr;
        if (cudaHostAlloc(&p, sizeof(uint32_t) * kGateStatusWords,
                          cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_gate_words = static_cast<uint32_t *>(p);
        g_gate_free = new std::vector<int>();
        for (int i = kGateStatusWords - 1; i >= 0; --i) g_gate_free->push_back(i);
    }
    if (g_gate_free->empty()) return nullptr;
    const int i = g_gate_free->back();
    g_gate_free->pop_back();
    return g_gate_words + i;
}

void gate_status_give(uint32_t *w) {
    if (!w) return;
    std::lock_guard<std::mutex> lk(g_gate_mu);
    g_gate_free->push_back(int(w - g_gate_words));
}

namespace {

// Poll interval of the gate (ns, approximate: __nanosleep sleeps up to
// twice this) and the longest wait a caller may ask for.
constexpr unsigned kGatePollNs = 1000;
constexpr uint64_t kGateMaxNs = 10ull * 1000 * 1000 * 1000;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread: wait until *flag >= target or the limit passes; status 1 =
// released, 2 = gave up.  Every iteration sleeps, so the iteration cap
// bounds the wait even if the global timer does not advance.
__global__ void gate_kernel(const volatile uint32_t *flag, uint32_t target, uint64_t timeout_ns,
                            uint64_t max_iter, volatile uint32_t *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t t0 = global_ns();
    uint32_t st = 2u;
    for (uint64_t it = 0; it < max_iter; ++it) {
        if (*flag >= target) {
            st = 1u;
            break;
        }
        if (global_ns() - t0 >= timeout_ns) break;
        __nanosleep(kGatePollNs);
    }
    *status = st;
    __threadfence_system();
}

}  // namespace
}  // namespace uccsd

extern "C" {

uccsd_status uccsd_gate_enqueue(uccsd_ctx *c, const uint32_t *flag, uint32_t target,
                                uint64_t timeout_ns, void *stream) {
    if (!c) return UCCSD_ERR_ARG;
    if (c->failed) {
        c->err = "context failed earlier: " + c->err;
        return UCCSD_ERR_STATE;
    }
    if (!flag || timeout_ns == 0 || timeout_ns > uccsd::kGateMaxNs) {
        c->err = "uccsd_gate_enqueue: null flag or a time limit outside (0, 10 s]";
        return UCCSD_ERR_ARG;
    }
    if (!stream) {
        c->err = "uccsd_gate_enqueue: the gate needs a non-default stream";
        return UCCSD_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess && !c->gate_status) {
        c->gate_status = uccsd::gate_status_take();
        if (!c->gate_status) {
            c->err = "uccsd_gate_enqueue: no gate status word left (pinned allocation failed or "
                     "4096 contexts hold gates)";
            return UCCSD_ERR_CUDA;
        }
    }
    if (e == cudaSuccess && !c->gate_ev) e = cudaEventCreateWithFlags(&c->gate_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        c->err = std::string("uccsd_gate_enqueue set-up: ") + cudaGetErrorString(e);
        return UCCSD_ERR_CUDA;
    }
    if (c->gate_pending && cudaEventQuery(c->gate_ev) == cudaErrorNotReady) {
        c->err = "uccsd_gate_enqueue: the context's previous gate is still waiting";
        return UCCSD_ERR_STATE;
    }
    cudaGetLastError();
    *reinterpret_cast<volatile uint32_t *>(c->gate_status) = 0u;
    uint32_t *status_dev = nullptr;
    e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&status_dev), c->gate_status, 0);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // iteration cap: the limit over the shortest poll, plus slack
    const uint64_t max_iter = timeout_ns / (uccsd::kGatePollNs / 4) + 1024;
    if (e == cudaSuccess) {
        uccsd::gate_kernel<<<1, 32, 0, s>>>(flag, target, timeout_ns, max_iter, status_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->gate_ev, s);
    if (e != cudaSuccess) {
        c->failed = true;
        c->err = std::string("uccsd_gate_enqueue: ") + cudaGetErrorString(e);
        return UCCSD_ERR_CUDA;
    }
    c->gate_pending = true;
    ++c->launches;
    return UCCSD_OK;
}

uccsd_status uccsd_gate_status(uccsd_ctx *c, int wait, int *released) {
    if (!c || !released) return UCCSD_ERR_ARG;
    *released = 0;
    if (!c->gate_pending) {
        c->err = "uccsd_gate_status: no gate enqueued";
        return UCCSD_ERR_STATE;
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = wait ? cudaEventSynchronize(c->gate_ev) : cudaEventQuery(c->gate_ev);
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return UCCSD_OK;  // still waiting
    }
    if (e != cudaSuccess) {
        c->failed = true;
        c->err = std::string("uccsd_gate_status: ") + cudaGetErrorString(e);
        return UCCSD_ERR_CUDA;
    }
    const uint32_t st = *reinterpret_cast<volatile uint32_t *>(c->gate_status);
    if (st == 1u) {
        *released = 1;
        return UCCSD_OK;
    }
    c->err = "uccsd_gate_status: the gate's time limit passed before the flag was released";
    return UCCSD_ERR_TIMEOUT;
}

uccsd_status uccsd_stream_mark(uccsd_ctx *c, void *stream) {
    if (!c || !stream) return UCCSD_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess && !c->mark_ev) e = cudaEventCreateWithFlags(&c->mark_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c->mark_ev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        c->err = std::string("uccsd_stream_mark: ") + cudaGetErrorString(e);
        return UCCSD_ERR_CUDA;
    }
    c->marked = true;
    return UCCSD_OK;
}

uccsd_status uccsd_mark_done(uccsd_ctx *c, int *done) {
    if (!c || !done) return UCCSD_ERR_ARG;
    if (!c->marked) {
        c->err = "uccsd_mark_done: no mark recorded";
        return UCCSD_ERR_STATE;
    }
    const cudaError_t e = cudaEventQuery(c->mark_ev);
    if (e == cudaSuccess || e == cudaErrorNotReady) {
        if (e == cudaErrorNotReady) cudaGetLastError();
        *done = e == cudaSuccess;
        return UCCSD_OK;
    }
    c->err = std::string("uccsd_mark_done: ") + cudaGetErrorString(e);
    return UCCSD_ERR_CUDA;
}

uccsd_status uccsd_zero_async(uccsd_ctx *c, void *ptr, size_t bytes, void *stream) {
    if (!c || !ptr) return UCCSD_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaMemsetAsync(ptr, 0, bytes, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        c->err = std::string("uccsd_zero_async: ") + cudaGetErrorString(e);
        return UCCSD_ERR_CUDA;
    }
    return UCCSD_OK;
}

}  // extern "C"
