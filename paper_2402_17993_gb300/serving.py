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
  its latency is arrival -> last step done.

The plain form (max_active = 1, use_graphs = False) steps one request at a
time from the host: evaluation, download, host L-BFGS update.

Fragments never share device buffers or reductions, so a fragment's result
does not depend on what else is in flight (checked by the GPU tests).
"""
from __future__ import annotations

import functools
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import FP32_STATE, FP64, Context, build_uccsd_list
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
    sector = math.comb(n_orb, n_alpha) * math.comb(n_orb, n_beta)  # adjoint hand-over vectors
    own = 2 * N * A + 2 * sector * A + K * tiles * 8 + K * 256 + tables
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


class _DevSlot:
    """A fragment whose whole solve is enqueued on its stream at admission:
    `steps` replays of one captured graph (evaluation + device L-BFGS step)."""

    def __init__(self, req, ctx, stream, t_admit, steps):
        import torch
        self.req = req
        self.ctx = ctx
        self.stream = stream
        self.K = ctx.K
        self.t_admit = t_admit
        self.steps = steps
        dev = torch.device("cuda", ctx.device)
        k = max(self.K, 1)
        ctx.opt_init(memory=10, max_step=0.2, first_scale=0.1, max_steps=steps)
        # everything of this fragment is ordered on its own stream
        with torch.cuda.stream(stream):
            buf = torch.zeros(2 * k + 1, dtype=torch.float64, device=dev)  # theta | grad | E
            self.th_dev, self.g_dev, self.E_dev = buf[:k], buf[k:2 * k], buf[2 * k:]
            ctx.capture_vqe_step(self.th_dev, self.E_dev, self.g_dev, stream)
            for _ in range(steps):
                ctx.replay(stream)  # evaluation + device L-BFGS step
            self.done = torch.cuda.Event()
            self.done.record(stream)

    def result(self, keep_theta):
        energies = [float(e) for e in self.ctx.opt_history(self.steps)]
        theta = self.th_dev[: self.K].cpu().numpy().copy() if keep_theta else None
        return energies, theta


class FragmentServer:
    """Serve fragment VQE solves with continuous batching on one GPU.

    precision: FP32_STATE (batched form) or FP64.  max_active = 1 with
    use_graphs = False gives the plain one-request-at-a-time form."""

    def __init__(self, precision=FP32_STATE, device=0, hbm_budget=8 << 30, max_active=48,
                 n_streams=None, steps=40, use_graphs=True):
        import torch
        self.precision = precision
        self.device = device
        self.hbm_budget = hbm_budget
        self.max_active = max_active
        self.steps = steps
        self.use_graphs = use_graphs
        n_streams = max_active if n_streams is None else n_streams
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self.pool = {}
        # pair lists held for each shape class seen (one shared copy per class)
        self.shared = {}

    def _context(self, req, used, stream=None):
        """A context for the request: a recycled one of the same shape class
        (its device buffers are reused, nothing is allocated) or a new one
        whose HBM budget is what the server has left.  With `stream` the
        set-up transfers are enqueued on it and nothing waits for them, so
        the host never stalls behind another fragment's solve."""
        key = (req.n_orb, req.n_alpha, req.n_beta)
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
        self.pool.setdefault((req.n_orb, req.n_alpha, req.n_beta), []).append(ctx)

    def close(self):
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
        }

    def _run_device(self, requests, rate, keep_theta):
        """Arrived requests are admitted in arrival order while slots and the
        HBM budget allow, one per pass of the loop between completion checks:
        the context is prepared with its set-up transfers enqueued on a free
        stream (host work, no host waits), then the evaluation graph is
        captured and the whole solve enqueued behind them on that stream."""
        reqs = sorted(requests, key=lambda q: q.t_unit)
        arrive = [0.0 if rate is None else q.t_unit / rate for q in reqs]
        t0 = time.perf_counter()
        pending = 0
        active: list[_DevSlot] = []
        free_streams = list(self.streams)
        results: list[Result] = []
        used = peak_used = sum(self.shared.values())
        dev_used = peak_dev = 0
        n_evals = 0
        while pending < len(reqs) or active:
            now = time.perf_counter() - t0
            progressed = False
            if (pending < len(reqs) and arrive[pending] <= now
                    and len(active) < self.max_active and free_streams):
                q = reqs[pending]
                need, extra = self._need(q)
                if used + need + extra <= self.hbm_budget or not active:
                    st = free_streams.pop()
                    ctx = self._context(q, used, st)
                    slot = _DevSlot(q, ctx, st, time.perf_counter() - t0, self.steps)
                    slot.reserved = need
                    slot.dev_bytes = ctx.info()["device_bytes"]
                    slot.t_arrive = arrive[pending]
                    if extra:
                        self.shared[(q.n_orb, q.n_alpha, q.n_beta)] = extra
                    used += need + extra
                    dev_used += slot.dev_bytes
                    peak_used = max(peak_used, used)
                    peak_dev = max(peak_dev, dev_used)
                    active.append(slot)
                    pending += 1
                    progressed = True
            still = []
            for s in active:
                if s.done.query():
                    t_done = time.perf_counter() - t0
                    energies, theta = s.result(keep_theta)
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
                if pending < len(reqs) and not active:
                    wait = max(0.0, min(arrive[pending] - (time.perf_counter() - t0), 0.01))
                time.sleep(wait)
        makespan = time.perf_counter() - t0
        stats = self._stats(results, n_evals, makespan, [], peak_used, peak_dev)
        # time average of the number of admitted, unfinished fragments
        stats["mean_active"] = (sum(r.t_done - r.t_admit for r in results) / makespan
                                if makespan > 0 else 0.0)
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


def fmo2_sum(monomer_E, dimer_E, n_frag):
    """Two-body FMO total (Eq. 1): sum over dimers minus (N_f - 2) times the
    sum over monomers."""
    return float(np.sum(dimer_E) - (n_frag - 2) * np.sum(monomer_E))


def capacity_rate(stats) -> float:
    """Requests per second the server sustained in a closed-loop run."""
    return stats["requests"] / stats["makespan_s"] if stats["makespan_s"] > 0 else math.inf
