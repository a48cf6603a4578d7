"""Continuous-batching server for a stream of FMO fragment VQE solves.

A two-body FMO job (Eq. 1 of the paper) needs one correlation solve per
monomer and per dimer; the paper ran them as separate jobs (Section 3.1).
Here requests arrive over time (monomers at 8-12 qubits, dimers at 16-18
qubits, each with its own integrals) and share one GPU:

* admission: a request enters when a slot is free and its device footprint
  (Hamiltonian tables, state and adjoint vectors, partial sums) fits the
  remaining HBM budget; the library enforces the same budget per context;
* residency: every admitted fragment keeps its context, state vectors and
  amplitudes on the device until its solve finishes;
* continuous batching: at admission a fragment's whole solve is enqueued on
  its own stream: a fixed number of steps, each one replay of its captured
  evaluation graph and one fixed-step L-BFGS update on the device
  (uccsd_opt_step), so no step waits for the host; solves of different
  fragments overlap on the device, and the host only admits arrivals into
  freed slots and collects finished solves;
* each solve runs a fixed number of optimiser steps (one evaluation each);
  its latency is arrival -> last step done;
* preparation off the serving thread: the host work of an admission (the
  Jordan-Wigner compile and tables, the sweep plans, the graph capture and
  the enqueue of the solve) runs on a pool of worker threads (8 by default),
  each on the fragment's own context and stream.  A context belongs to one thread at a
  time: the pool hands it to a worker, the worker hands the prepared
  fragment to the serving thread, and the serving thread returns the
  context to the pool only after it has read the results (the library's
  contexts are independent of each other, but not thread-safe each).

The plain form (max_active = 1, use_graphs = False) steps one request at a
time from the host: evaluation, download, host L-BFGS update.

Fragments never share device buffers or reductions, so a fragment's result
does not depend on what else is in flight (checked by the GPU tests).
"""
from __future__ import annotations

import bisect
import functools
import math
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import FP32_STATE, FP64, Context, UCCSDError, build_uccsd_list
from .vqe import LBFGS


@dataclass
class Request:
    r: int
    t_unit: float     # arrival time at unit rate (seconds = t_unit / rate)
    n_orb: int
    n_alpha: int
    n_beta: int
    h: np.ndarray     # (n_orb, n_orb) one-electron integrals
    eri: np.ndarray   # (n_orb,)*4 chemist-notation two-electron integrals
    e_core: float = 0.0

    @property
    def n_elec(self):
        return self.n_alpha + self.n_beta


@dataclass
class Result:
    r: int
    n_qubits: int
    t_arrive: float
    t_admit: float
    t_done: float
    energy: float
    energies: list = field(default_factory=list)
    theta: np.ndarray | None = None

    @property
    def latency(self):
        return self.t_done - self.t_arrive


@functools.lru_cache(maxsize=None)
def list_bytes(n_orb: int, n_alpha: int, n_beta: int) -> int:
    """Upper estimate of the precomputed pair lists of one shape class
    (bytes): the pairs of each excitation on the whole sector (exact for
    one-tile plans), for the forward plan and up to twice that for the
    adjoint plan, 8 bytes per pair.  One device copy serves every context of
    the class."""
    from math import comb
    pairs = 0
    for i, j, a, b in build_uccsd_list(n_orb, n_alpha, n_beta).tolist():
        na = sum(1 for q in (i, j, a, b) if q >= 0 and q % 2 == 0) // 2
        nb = sum(1 for q in (i, j, a, b) if q >= 0 and q % 2 == 1) // 2
        pairs += (comb(n_orb - 2 * na, n_alpha - na) * comb(n_orb - 2 * nb, n_beta - nb))
    return 3 * 8 * pairs


@functools.lru_cache(maxsize=None)
def footprint_bytes(n_orb: int, n_alpha: int, n_beta: int, precision: int,
                    lists: bool = True) -> int:
    """Upper estimate of one context's device memory (bytes); lists=False
    leaves out the pair lists shared within the shape class."""
    n = 2 * n_orb
    N = 1 << n
    A = 8 if precision == FP32_STATE else 16
    K = len(build_uccsd_list(n_orb, n_alpha, n_beta))
    tiles = max(1, N >> 10)
    tables = 200 * (n_orb ** 4) + (4 << 20)
    # compact sector vectors: psi and sigma between the kernels, phi and
    # lambda between the adjoint's runs
    sector = math.comb(n_orb, n_alpha) * math.comb(n_orb, n_beta)
    own = 2 * N * A + 4 * sector * A + K * tiles * 8 + K * 256 + tables
    return own + (list_bytes(n_orb, n_alpha, n_beta) if lists else 0)


class _Slot:
    def __init__(self, req, ctx, precision, stream, t_admit, steps):
        import torch
        self.req = req
        self.ctx = ctx
        self.stream = stream
        self.K = ctx.K
        self.t_admit = t_admit
        self.steps_left = steps
        self.theta = np.zeros(self.K)
        self.opt = LBFGS(self.K)
        dev = torch.device("cuda", ctx.device)
        self.th_dev = torch.zeros(max(self.K, 1), dtype=torch.float64, device=dev)
        self.E_dev = torch.zeros(1, dtype=torch.float64, device=dev)
        self.g_dev = torch.zeros(max(self.K, 1), dtype=torch.float64, device=dev)
        self.th_host = torch.zeros(max(self.K, 1), dtype=torch.float64).pin_memory()
        self.out_host = torch.zeros(1 + max(self.K, 1), dtype=torch.float64).pin_memory()
        self.event = torch.cuda.Event()
        self.energies = []
        self.used_graph = False

    def launch(self, use_graph: bool):
        import torch
        with torch.cuda.stream(self.stream):
            self.th_host[: self.K] = torch.from_numpy(self.theta)
            self.th_dev.copy_(self.th_host, non_blocking=True)
            if use_graph:
                if not self.used_graph:
                    self.ctx.capture(self.th_dev[: self.K].view(1, -1), self.E_dev,
                                     self.g_dev[: self.K].view(1, -1), self.stream)
                    self.used_graph = True
                self.ctx.replay(self.stream)
            else:
                self.ctx.energy_grad_device(self.th_dev[: self.K].view(1, -1), self.E_dev,
                                            self.g_dev[: self.K].view(1, -1), self.stream)
            self.out_host[0:1].copy_(self.E_dev, non_blocking=True)
            self.out_host[1: 1 + self.K].copy_(self.g_dev[: self.K], non_blocking=True)
            self.event.record(self.stream)

    def finish_step(self):
        self.event.synchronize()
        E = float(self.out_host[0])
        g = self.out_host[1: 1 + self.K].numpy().copy()
        self.energies.append(E)
        self.steps_left -= 1
        if self.steps_left > 0 and self.K > 0:
            self.theta = self.opt.step(self.theta, g)
        return E


class _Mark:
    """Completion of a fragment's enqueued solve (the context's stream mark),
    queried without waiting."""

    def __init__(self, ctx):
        self.ctx = ctx

    def query(self):
        return self.ctx.mark_done()


class _DevSlot:
    """A fragment whose whole solve is enqueued on its stream at admission:
    `steps` replays of one captured graph (evaluation + device L-BFGS step)."""

    def __init__(self, req, ctx, stream, t_admit, steps, gate_flag=None, gate_timeout_s=5.0,
                 buf=None):
        import torch
        self.req = req
        self.ctx = ctx
        self.stream = stream
        self.K = ctx.K
        self.t_admit = t_admit
        self.steps = steps
        self.gate_flag = gate_flag
        self.buf = buf
        dev = torch.device("cuda", ctx.device)
        k = max(self.K, 1)
        ctx.opt_init(memory=10, max_step=0.2, first_scale=0.1, max_steps=steps)
        # Everything of this fragment is ordered on its own stream, and every
        # enqueue goes through the library: a launch may wait in the driver
        # while a hardware queue is full of solves held by gates, and a plain
        # C call lets the serving thread run meanwhile to release them.
        if buf is None:
            buf = torch.empty(2 * k + 1, dtype=torch.float64, device=dev)  # theta | grad | E
        buf = buf[: 2 * k + 1]
        ctx.zero_async(buf, stream)  # theta starts at zero
        self.th_dev, self.g_dev, self.E_dev = buf[:k], buf[k:2 * k], buf[2 * k:]
        ctx.capture_vqe_step(self.th_dev, self.E_dev, self.g_dev, stream)
        if gate_flag is not None:
            # prepared ahead of its arrival: the solve waits on the device
            # until the serving thread releases the flag
            ctx.gate(gate_flag, 1, gate_timeout_s, stream)
        for _ in range(steps):
            ctx.replay(stream)  # evaluation + device L-BFGS step
        ctx.mark(stream)
        self.done = _Mark(ctx)

    def release(self):
        self.gate_flag[0] = 1

    def check_gate(self):
        """False if the gate gave up before its release: the solve then ran
        early (its result is the same, its latency is void)."""
        if self.gate_flag is None:
            return True
        try:
            return self.ctx.gate_status(wait=True)
        except UCCSDError as exc:
            if exc.code != 5:  # anything but the gate's own time limit
                raise
            return False

    def result(self, keep_theta):
        energies = [float(e) for e in self.ctx.opt_history(self.steps)]
        theta = self.th_dev[: self.K].cpu().numpy().copy() if keep_theta else None
        return energies, theta


class FragmentServer:
    """Serve fragment VQE solves with continuous batching on one GPU.

    precision: FP32_STATE (batched form) or FP64.  max_active = 1 with
    use_graphs = False gives the plain one-request-at-a-time form."""

    def __init__(self, precision=FP32_STATE, device=0, hbm_budget=8 << 30, max_active=48,
                 n_streams=None, steps=40, use_graphs=True, prep_workers=8, lookahead=0):
        import torch
        self.precision = precision
        self.device = device
        self.hbm_budget = hbm_budget
        self.max_active = max_active
        self.steps = steps
        self.use_graphs = use_graphs
        n_streams = max_active if n_streams is None else n_streams
        self.streams = _distinct_streams(device, n_streams)
        # Streams beyond the device's hardware work queues share queues and
        # serialise falsely (the default is 8 queues: the closed-loop stream
        # runs at about 11K instead of 38K evaluations/s with 32 streams).
        # The queue count is read when CUDA initialises, so the process sets
        # CUDA_DEVICE_MAX_CONNECTIONS before that (bench.py sets 32).
        import os
        import warnings
        conn = int(os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"))
        if conn < min(len(self.streams), 32):
            warnings.warn(f"CUDA_DEVICE_MAX_CONNECTIONS={conn} hardware queues for "
                          f"{len(self.streams)} fragment streams: set it (to 32) before CUDA "
                          "initialises, or fragments on shared queues serialise", RuntimeWarning)
        self.pool = {}
        self._pool_lock = threading.Lock()
        # pair lists held for each shape class seen (one shared copy per class)
        self.shared = {}
        # host threads that prepare admitted fragments (0: the serving thread)
        self.prep_workers = prep_workers
        self._exec = (ThreadPoolExecutor(prep_workers, thread_name_prefix="uccsd-prep")
                      if prep_workers > 0 and use_graphs else None)
        # requests prepared before their arrival, each behind a device gate
        # that the serving thread releases at the arrival (open-loop runs)
        self.lookahead = lookahead

    def _context(self, req, used, stream=None):
        """A context for the request: a recycled one of the same shape class
        (its device buffers are reused, nothing is allocated) or a new one
        whose HBM budget is what the server has left.  With `stream` the
        set-up transfers are enqueued on it and nothing waits for them, so
        the host never stalls behind another fragment's solve."""
        key = (req.n_orb, req.n_alpha, req.n_beta)
        with self._pool_lock:
            pool = self.pool.get(key)
            ctx = pool.pop() if pool else None
        if ctx is None:
            ctx = Context(self.device, self.precision, max(1, self.hbm_budget - used))
        ctx.set_setup_stream(stream)
        ctx.set_hamiltonian(req.n_orb, req.h, req.eri, req.e_core)
        ctx.set_reference(req.n_alpha, req.n_beta)
        ctx.set_excitations(build_uccsd_list(req.n_orb, req.n_alpha, req.n_beta))
        return ctx

    def _need(self, req):
        """(per-request reservation, shared pair-list bytes still to reserve
        for the request's shape class)."""
        key = (req.n_orb, req.n_alpha, req.n_beta)
        need = footprint_bytes(*key, self.precision, lists=False)
        return need, (0 if key in self.shared else list_bytes(*key))

    def _release(self, req, ctx):
        with self._pool_lock:
            self.pool.setdefault((req.n_orb, req.n_alpha, req.n_beta), []).append(ctx)

    def _prepare(self, q, used, stream, t0, gate_flag=None, buf=None):
        """Host work of one admission (on a worker thread or the serving
        thread): the context's set-up on the fragment's stream, then the
        capture of its evaluation and optimiser step and the enqueue of the
        whole solve (behind a gate when it is prepared ahead of arrival)."""
        import torch
        torch.cuda.set_device(self.device)
        ctx = self._context(q, used, stream)
        slot = _DevSlot(q, ctx, stream, time.perf_counter() - t0, self.steps, gate_flag, buf=buf)
        slot.dev_bytes = ctx.info()["device_bytes"]
        return slot

    def close(self):
        if self._exec is not None:
            self._exec.shutdown(wait=True)
            self._exec = None
        for lst in self.pool.values():
            for ctx in lst:
                ctx.close()
        self.pool = {}
        self.shared = {}

    def run(self, requests, rate=None, keep_theta=False):
        """Serve `requests` (arrivals at t_unit / rate seconds; rate None =
        all at once).  Returns (results, stats)."""
        if self.use_graphs:
            return self._run_device(requests, rate, keep_theta)
        return self._run_host(requests, rate, keep_theta)

    def _stats(self, results, n_evals, makespan, active_hist, peak_used, peak_dev):
        lat = np.array([r.latency for r in results])
        return {
            "requests": len(results), "steps_per_solve": self.steps, "evals": n_evals,
            "makespan_s": makespan, "evals_per_s": n_evals / makespan,
            "p50_latency_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_latency_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "mean_active": float(np.mean(active_hist)) if active_hist else 0.0,
            "peak_hbm_reserved_bytes": int(peak_used),
            "peak_hbm_device_bytes": int(peak_dev),
            "precision": "fp32" if self.precision == FP32_STATE else "fp64",
            "max_active": self.max_active, "graphs": self.use_graphs,
            "streams": len(self.streams),
        }

    def _run_device(self, requests, rate, keep_theta):
        """Arrived requests are admitted in arrival order while slots, streams
        and the HBM budget allow; each admission reserves its budget and a
        free stream on the serving thread and hands the host work (context
        set-up, capture, enqueue of the whole solve on that stream) to a
        worker thread.  The serving thread collects prepared fragments and
        finished solves."""
        import torch
        reqs = sorted(requests, key=lambda q: q.t_unit)
        arrive = [0.0 if rate is None else q.t_unit / rate for q in reqs]
        t0 = time.perf_counter()
        pending = 0
        active: list[_DevSlot] = []
        preparing = []  # (future, request, reserved bytes, arrival time)
        gated = []      # (arrival time, gate flag) not yet released, in arrival order
        release_lag = 0.0   # longest delay between an arrival and its gate's release
        gates_gave_up = 0
        # Gate flags, pinned once before the loop: while gates wait on the
        # device, the serving thread must make no call that waits for the
        # device (a pinned allocation may), or it waits for the gates that
        # only it can release, until their time limit.
        n_flags = self.max_active + 1
        flag_buf = torch.zeros(n_flags, dtype=torch.int32).pin_memory() if rate and self.lookahead else None
        free_flags = list(range(n_flags))
        # For the same reason the solves' device buffers (theta | grad | E) are
        # allocated here: a device allocation on a preparing worker thread
        # waits for the device while holding the interpreter lock, which the
        # serving thread then cannot take to release the gates.
        slot_bufs = []
        if flag_buf is not None:
            kmax = max(max(1, len(build_uccsd_list(q.n_orb, q.n_alpha, q.n_beta))) for q in reqs)
            dev = torch.device("cuda", self.device)
            slot_bufs = [torch.zeros(2 * kmax + 1, dtype=torch.float64, device=dev)
                         for _ in range(self.max_active)]
            torch.cuda.synchronize(dev)
        free_streams = list(self.streams)
        results: list[Result] = []
        used = peak_used = sum(self.shared.values())
        dev_used = peak_dev = 0
        n_evals = 0
        while pending < len(reqs) or active or preparing:
            now = time.perf_counter() - t0
            progressed = False
            # requests up to `lookahead` past the arrived ones are prepared
            # early, behind a gate
            n_arrived = bisect.bisect_right(arrive, now)
            while (pending < len(reqs) and pending < n_arrived + (self.lookahead if rate else 0)
                   and len(active) + len(preparing) < self.max_active and free_streams):
                q = reqs[pending]
                need, extra = self._need(q)
                if used + need + extra > self.hbm_budget and (active or preparing):
                    break
                st = free_streams.pop()
                if extra:
                    self.shared[(q.n_orb, q.n_alpha, q.n_beta)] = extra
                before = used  # the context's own budget: what the others leave
                used += need + extra
                peak_used = max(peak_used, used)
                flag = None
                if arrive[pending] > now and flag_buf is not None:
                    fi = free_flags.pop()
                    flag = flag_buf[fi:fi + 1]
                    flag[0] = 0
                    gated.append((arrive[pending], flag))
                sbuf = slot_bufs.pop() if slot_bufs else None
                if self._exec is not None:
                    fut = self._exec.submit(self._prepare, q, before, st, t0, flag, sbuf)
                else:
                    fut = _Done(self._prepare(q, before, st, t0, flag, sbuf))
                preparing.append((fut, q, need, arrive[pending]))
                pending += 1
                progressed = True
                if self._exec is None:
                    break  # one admission per pass when the serving thread prepares
            # release the gates of the requests that have arrived
            now = time.perf_counter() - t0
            while gated and gated[0][0] <= now:
                t_arr, flag = gated.pop(0)
                flag[0] = 1
                release_lag = max(release_lag, now - t_arr)
                progressed = True
            still_prep = []
            for fut, q, need, t_arr in preparing:
                if fut.done():
                    slot = fut.result()
                    slot.reserved = need
                    slot.t_arrive = t_arr
                    dev_used += slot.dev_bytes
                    peak_dev = max(peak_dev, dev_used)
                    active.append(slot)
                    progressed = True
                else:
                    still_prep.append((fut, q, need, t_arr))
            preparing = still_prep
            still = []
            for s in active:
                if s.done.query():
                    t_done = time.perf_counter() - t0
                    if not s.check_gate():
                        gates_gave_up += 1
                    if s.gate_flag is not None:
                        free_flags.append((s.gate_flag.data_ptr() - flag_buf.data_ptr()) // 4)
                    energies, theta = s.result(keep_theta)
                    if s.buf is not None:  # free again once its results are read
                        slot_bufs.append(s.buf)
                    results.append(Result(s.req.r, 2 * s.req.n_orb, s.t_arrive, s.t_admit,
                                          t_done, energies[-1], energies, theta))
                    n_evals += s.steps
                    used -= s.reserved
                    dev_used -= s.dev_bytes
                    free_streams.append(s.stream)
                    self._release(s.req, s.ctx)
                    progressed = True
                else:
                    still.append(s)
            active = still
            if not progressed:
                wait = 50e-6
                if pending < len(reqs) and not active and not preparing and not gated:
                    wait = max(0.0, min(arrive[pending] - (time.perf_counter() - t0), 0.01))
                time.sleep(wait)
        makespan = time.perf_counter() - t0
        stats = self._stats(results, n_evals, makespan, [], peak_used, peak_dev)
        stats["lookahead"] = self.lookahead if rate else 0
        if stats["lookahead"]:
            stats["max_gate_release_lag_ms"] = 1e3 * release_lag
            stats["gates_gave_up"] = gates_gave_up
        # time average of the number of admitted, unfinished fragments
        stats["mean_active"] = (sum(r.t_done - r.t_admit for r in results) / makespan
                                if makespan > 0 else 0.0)
        stats["prep_workers"] = self.prep_workers if self._exec is not None else 0
        return sorted(results, key=lambda r: r.r), stats

    def _run_host(self, requests, rate, keep_theta):
        reqs = sorted(requests, key=lambda q: q.t_unit)
        arrive = [0.0 if rate is None else q.t_unit / rate for q in reqs]
        t0 = time.perf_counter()
        pending = 0
        active: list[_Slot] = []
        results: list[Result] = []
        used = sum(self.shared.values())  # reserved by admission (upper estimates)
        peak_used = used
        dev_used = 0      # device bytes the active contexts report
        peak_dev = 0
        n_evals = 0
        active_hist = []
        next_stream = 0
        while pending < len(reqs) or active:
            now = time.perf_counter() - t0
            # admission: FIFO over arrived requests while slots and HBM allow
            while (pending < len(reqs) and arrive[pending] <= now
                   and len(active) < self.max_active):
                q = reqs[pending]
                need, extra = self._need(q)
                if used + need + extra > self.hbm_budget and active:
                    break
                if extra:
                    self.shared[(q.n_orb, q.n_alpha, q.n_beta)] = extra
                used += extra
                ctx = self._context(q, used)
                slot = _Slot(q, ctx, self.precision, self.streams[next_stream % len(self.streams)],
                             now, self.steps)
                slot.reserved = need
                slot.dev_bytes = ctx.info()["device_bytes"]
                slot.t_arrive = arrive[pending]
                next_stream += 1
                used += need
                dev_used += slot.dev_bytes
                peak_used = max(peak_used, used)
                peak_dev = max(peak_dev, dev_used)
                active.append(slot)
                pending += 1
            if not active:
                time.sleep(max(0.0, min(arrive[pending] - (time.perf_counter() - t0), 0.01)))
                continue
            active_hist.append(len(active))
            for s in active:
                s.launch(self.use_graphs)
            still = []
            for s in active:
                s.finish_step()
                n_evals += 1
                if s.steps_left <= 0:
                    t_done = time.perf_counter() - t0
                    results.append(Result(s.req.r, 2 * s.req.n_orb, s.t_arrive, s.t_admit, t_done,
                                          s.energies[-1], s.energies,
                                          s.theta.copy() if keep_theta else None))
                    used -= s.reserved
                    dev_used -= s.dev_bytes
                    self._release(s.req, s.ctx)
                else:
                    still.append(s)
            active = still
        makespan = time.perf_counter() - t0
        return (sorted(results, key=lambda r: r.r),
                self._stats(results, n_evals, makespan, active_hist, peak_used, peak_dev))


def _distinct_streams(device, n):
    """Up to n CUDA streams with distinct handles.  torch.cuda.Stream() draws
    from a fixed pool (32 streams per priority), so asking for more repeats
    handles; two fragments on one handle would share a stream (their solves
    serialise), and a capture on it by one preparing thread would collide
    with another thread's launches.  All at the default priority, so no
    fragment is preferred: the server then runs at most as many fragments at
    once as there are distinct streams."""
    import torch
    seen, out = set(), []
    for _ in range(2 * n + 64):
        st = torch.cuda.Stream(device=device)
        if st.cuda_stream not in seen:
            seen.add(st.cuda_stream)
            out.append(st)
            if len(out) == n:
                break
    return out


class _Done:
    """A finished result in the shape of a future (preparation on the
    serving thread)."""

    def __init__(self, value):
        self.value = value

    def done(self):
        return True

    def result(self):
        return self.value


def fmo2_sum(monomer_E, dimer_E, n_frag):
    """Two-body FMO total (Eq. 1): sum over dimers minus (N_f - 2) times the
    sum over monomers."""
    return float(np.sum(dimer_E) - (n_frag - 2) * np.sum(monomer_E))


def fmo_fragment_integrals(h, eri, frag_orbs, frag_nocc, members):
    """Integrals of a monomer (members = (I,)) or dimer ((I, J)) of a
    supersystem in localised orbitals (Section 2.1): the members' orbitals,
    ordered [occupied of each member, then virtual of each member] so that
    the reference determinant is the lowest orbitals, with the one-electron
    part embedded in the mean field of the other fragments' closed-shell
    reference determinants,
        h_pq + sum_{j occupied in the environment} (2 (pq|jj) - (pj|jq)).
    Returns (h, eri, n_occ) with n_occ = occupied spatial orbitals."""
    occ = [o for f in members for o in frag_orbs[f][:frag_nocc[f]]]
    vir = [o for f in members for o in frag_orbs[f][frag_nocc[f]:]]
    sel = np.array(occ + vir)
    env = np.array([o for f in range(len(frag_orbs)) if f not in members
                    for o in frag_orbs[f][:frag_nocc[f]]], dtype=int)
    hs = h[np.ix_(sel, sel)].copy()
    if env.size:
        coul = eri[np.ix_(sel, sel, env, env)]
        exch = eri[np.ix_(sel, env, env, sel)]
        hs += 2.0 * np.einsum("pqjj->pq", coul) - np.einsum("pjjq->pq", exch)
    es = np.ascontiguousarray(eri[np.ix_(sel, sel, sel, sel)])
    return np.ascontiguousarray(0.5 * (hs + hs.T)), es, len(occ)


def fmo2_requests(h, eri, frag_orbs, frag_nocc):
    """Requests of a two-body FMO job: every monomer and every dimer of the
    supersystem (Eq. 1 needs E_I and E_IJ).  Returns (requests, keys) with
    keys[i] = the members of request i."""
    n_frag = len(frag_orbs)
    keys = [(i,) for i in range(n_frag)] + [(i, j) for i in range(n_frag)
                                             for j in range(i + 1, n_frag)]
    reqs = []
    for r, key in enumerate(keys):
        hf, ef, nocc = fmo_fragment_integrals(h, eri, frag_orbs, frag_nocc, key)
        reqs.append(Request(r, 0.0, hf.shape[0], nocc, nocc, hf, ef, 0.0))
    return reqs, keys


def fmo2_total(energies, keys, n_frag):
    """Eq. 1 from the energies of fmo2_requests' fragments (same order)."""
    mono = [e for e, k in zip(energies, keys) if len(k) == 1]
    dim = [e for e, k in zip(energies, keys) if len(k) == 2]
    return fmo2_sum(mono, dim, n_frag)


def capacity_rate(stats) -> float:
    """Requests per second the server sustained in a closed-loop run."""
    return stats["requests"] / stats["makespan_s"] if stats["makespan_s"] > 0 else math.inf
