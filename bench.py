#!/usr/bin/env python
"""Benchmark: Trotterised UCCSD energy + adjoint-gradient evaluations per
second on GB300 (sm_103a), one JSON line on stdout.

Workload (one step): the 18-qubit dimer-scale fragment (10 electrons, 9
spatial orbitals, synthetic integrals seed 2 with 16 Cholesky vectors,
K = 560 spin-conserving singles+doubles, first-order Trotter, M = 1) with a
batch of 64 amplitude vectors theta ~ N(0, 0.05) (seeds 1002+b): one energy
and full gradient per vector, FP32 state with FP64 reductions.  The
26-qubit scale-up (12 electrons, K = 2478, seed 4) is timed as well and
reported under "scaleup".

--impl reference times the CPU oracle (FP64, OpenMP on the host cores) on
a bounded sample of the same workload.

Under torchrun each rank evaluates its own batch of 64 (weak scaling; the
evaluations are independent, there is no data-path collective).
"""
from __future__ import annotations

import os

# one CUDA stream per active fragment in the serving measurement: allow more
# hardware work queues than the default 8 (read when CUDA initialises)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "UCCSD energy+grad evals/s (18q dimer fragment, batch 64)"
METRIC_26Q = "UCCSD energy+grad evals/s (26q scale-up, one state)"
WORKLOAD_26Q = ("26q/12e UCCSD K=2478 (seed 4, 20 Cholesky), theta ~N(0,0.02) (seeds 1004+b), "
                "energy+adjoint gradient, M=1 first-order Trotter")
WORKLOAD = ("18q/10e UCCSD K=560 (seed 2, 16 Cholesky), batch 64 theta ~N(0,0.05), "
            "energy+adjoint gradient, M=1 first-order Trotter")
UNIT = "evals/s"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=None,
                    help="states per step (default 64 at 18 qubits, 1 at 26 qubits)")
    ap.add_argument("--workload", default="18q", choices=["18q", "26q"],
                    help="timed workload: the 18-qubit dimer batch (the headline) or the "
                         "26-qubit scale-up")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--layout", default="full", choices=["full", "sector"],
                    help="state layout of the timed path (the sector layout is also timed "
                         "beside the full one as a comparison)")
    ap.add_argument("--no-layout-compare", action="store_true")
    ap.add_argument("--no-scaleup", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the 8- and 12-qubit workloads (sweep, VQE)")
    ap.add_argument("--serving-requests", type=int, default=512)
    ap.add_argument("--serving-fp64-requests", type=int, default=None,
                    help="requests of the one-at-a-time FP64 arm (default: the same stream "
                         "as the batched arm)")
    args = ap.parse_args()
    if args.batch is None:
        args.batch = 64 if args.workload == "18q" else 1
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, world: int) -> float:
    """Max of x over the ranks (the job's timed region ends with its slowest
    rank).  Uses the process group's backend: NCCL on GPUs, gloo on CPUs."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Weak scaling: every rank evaluates its own units (no data-path
    collective); the job rate is all ranks' units over the slowest rank's
    time."""
    return world * units_per_rank / (max_ms / 1e3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class NvmlClocks:
    """SM clock, its maximum and the clock-event reasons of one GPU, read
    through NVML (libnvidia-ml, read-only queries) every 10 ms by a host
    thread while the timed region runs, so even a short region gets many
    samples.  The GPU is found by its PCI bus id (as CUDA numbers it)."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, device):
        import ctypes
        import threading
        self._ct = ctypes
        self.nv = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(device)
            bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        except Exception:
            bus = None
        ok = bus is not None and self.nv.nvmlDeviceGetHandleByPciBusId_v2(
            bus.encode(), ctypes.byref(self.h)) == 0
        if not ok and self.nv.nvmlDeviceGetHandleByIndex_v2(device, ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        try:
            self._reasons_fn = self.nv.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self._reasons_fn = self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples = []
        self.reasons = 0
        self.stop_ev = threading.Event()
        self.th = threading.Thread(target=self._run, daemon=True)

    def _read(self):
        ct = self._ct
        mhz = ct.c_uint()
        rs = ct.c_ulonglong()
        if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) == 0:  # NVML_CLOCK_SM
            self.samples.append(mhz.value)
        if self._reasons_fn(self.h, ct.byref(rs)) == 0:
            self.reasons |= rs.value

    def _run(self):
        while not self.stop_ev.is_set():
            self._read()
            self.stop_ev.wait(0.01)

    def start(self):
        self.th.start()

    def stop(self):
        self.stop_ev.set()
        self.th.join()
        self._read()
        mx = self._ct.c_uint()
        smax = (float(mx.value) if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, self._ct.byref(mx)) == 0
                else None)
        self.nv.nvmlShutdown()
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                "sm_max_mhz": smax,
                "reasons": sorted(v for b, v in self.REASONS.items() if self.reasons & b),
                "samples": len(self.samples), "source": "NVML every 10 ms"}


def clock_sampler(device):
    """NVML sampler where libnvidia-ml loads, else nvidia-smi every 200 ms."""
    try:
        return NvmlClocks(device)
    except Exception:
        return Clocks(device)


class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi every 200 ms"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# oracle arm
# ---------------------------------------------------------------------------
def oracle_rate(w, thetas, n_eval):
    import oracle
    ex = oracle.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
    t = time.perf_counter()
    for b in range(n_eval):
        oracle.energy_grad(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                           ex, thetas[b % len(thetas)], sector=True)
    dt = time.perf_counter() - t
    return n_eval / dt, dt, oracle.num_threads()


def oracle_rate_single_thread(seed: int = 1002) -> float:
    """The oracle's rate on one host core: one 18-qubit evaluation in a
    child process started with OMP_NUM_THREADS=1 (OpenMP reads it once, at
    start-up)."""
    code = ("import sys, time; sys.path.insert(0, %r); import oracle, synth; "
            "w = synth.workload('18q'); "
            "ex = oracle.excitations(w['n_orb'], w['n_alpha'], w['n_beta']); "
            "th = synth.theta_normal(len(ex), 0.05, %d); t = time.perf_counter(); "
            "oracle.energy_grad(w['n_orb'], w['h'], w['eri'], w['e_core'], w['n_alpha'], "
            "w['n_beta'], ex, th, sector=True); "
            "print(time.perf_counter() - t, oracle.num_threads())") % (ROOT, seed)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    dt, threads = out.stdout.split()[-2:]
    if int(threads) != 1:
        raise RuntimeError("the oracle did not run on one thread")
    return 1.0 / float(dt)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = synth.workload("18q")
    K = 560
    thetas = [synth.theta_normal(K, 0.05, 1002 + b) for b in range(args.batch)]
    per_step = 4
    for _ in range(args.warmup):
        oracle_rate(w, thetas, 1)
    t = time.perf_counter()
    for s in range(args.steps):
        oracle_rate(w, thetas[(s * per_step) % args.batch:], per_step)
    dt = time.perf_counter() - t
    value = args.steps * per_step / dt
    sample = f"{per_step} of the 64 theta vectors per step (sector-restricted FP64 oracle)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
KERNEL_SOURCES = {"happly": "kernels.cu", "forward": "sweep.cu", "adjoint": "sweep.cu"}
FP64_PEAK_TFLOPS = 1.25  # GB300's nominal FP64 rate (no measured figure exists)


def device_peaks(sm_count, sm_max_mhz):
    """Peaks of the bounds that no measured figure covers, derived from the
    device's SM count and maximum SM clock (both read at run time):
      FP32 ALU: SMs x 128 FP32 lanes x 2 flops (FMA) per clock;
      shared memory: SMs x 32 banks x 4 bytes per clock."""
    hz = sm_max_mhz * 1e6
    return {"fp32_tflops": sm_count * 128 * 2 * hz / 1e12,
            "smem_gbs": sm_count * 128 * hz / 1e9,
            "sm_count": sm_count, "sm_max_mhz": sm_max_mhz}


def full_space_work(fam, n, amp_bytes, ijab, n_groups):
    """The same work counted over all 2^n amplitudes (active-pair bytes of
    every factor; one update per X-mask group and amplitude).  The kernels
    never touch the amplitudes outside the electron sector, so this is an
    equivalent rate, not a fraction of any peak."""
    N = 1 << n
    singles = int(np.sum(ijab[:, 1] < 0))
    doubles = len(ijab) - singles
    fwd = 2.0 * amp_bytes * N * (singles / 2 + doubles / 8)
    return {"forward": (fwd, "bytes"), "adjoint": (2.0 * fwd, "bytes"),
            "happly": (4.0 * n_groups * N, "flops")}.get(fam, (0.0, None))


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary of this kernel
    and workload, if the kernel source is unchanged since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    src = os.path.join(ROOT, "paper_2402_17993_gb300", "csrc", KERNEL_SOURCES.get(kernel, ""))
    if not os.path.exists(path) or not os.path.exists(src):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    rec_sha, traffic = None, None
    for line in open(path):
        if line.startswith("kernel source sha256:"):
            rec_sha = line.split(":", 1)[1].strip()
        if line.startswith("| DRAM traffic per launch (read + write) |"):
            traffic = float(line.split("|")[2].split()[0])
    return traffic if rec_sha == sha else None


def sector_bytes(fam, info, amp_bytes, B):
    """Compulsory HBM bytes of one evaluation call of a kernel family on
    the electron sector (D = C(n_orb, n_alpha) C(n_orb, n_beta) amplitudes
    per state): the forward writes psi once per run and reads it back in
    every later run; the H-apply reads psi and writes sigma; the adjoint
    reads phi and lambda once per run and writes them for every run but
    the last."""
    from math import comb
    D = comb(info["n_qubits"] // 2, info["n_alpha"]) * comb(info["n_qubits"] // 2, info["n_beta"])
    v = D * amp_bytes * B
    if fam == "forward":
        return v * (2 * info["n_fwd_runs"] - 1)
    if fam == "happly":
        return 2 * v
    if fam == "adjoint":
        return 2 * v * (2 * info["n_adj_runs"] - 1)
    return 0


def roofline(prof, B, info, amp_bytes, ijab, prec_fp32, workload, dev_pk):
    """Per kernel family: its algorithmic work on the electron sector, the
    rate over the CUDA-event launch time and the fraction of the peak that
    bounds it.
      happly   4 flops per connected group contribution of every sector
               amplitude, against the FP32 (FP64) ALU peak;
      forward  the sector's active pairs of every factor, 2 loads + 2 stores
               per pair, against the shared-memory peak (the tile stays in
               shared memory through a run);
      adjoint  the same for phi and lambda."""
    pk, pk_kind = peaks()
    n, na, nb = info["n_qubits"], info["n_alpha"], info["n_beta"]
    fams = {}
    for fam in ("forward", "happly", "adjoint"):
        if prof["launches"][fam] == 0:
            continue
        calls = max(1, prof["calls"])
        ms = prof["ms"][fam] / calls                      # device time per evaluation call
        launches = prof["launches"][fam] / calls
        if fam == "happly":
            work = sector_updates_per_state(n // 2, na, nb) * 4.0 * B
            peak = dev_pk["fp32_tflops"] if prec_fp32 else FP64_PEAK_TFLOPS
            achieved, unit, bound = work / (ms / 1e3) / 1e12, "TFLOP/s", "alu"
            basis = ("4 flops per connected group contribution of each electron-sector "
                     "amplitude (the diagonal, same-spin singles and doubles, mixed doubles)")
            peak_kind = ("derived: SMs x 128 FP32 lanes x 2 x max SM clock" if prec_fp32
                         else "nominal FP64")
        else:
            vecs = 1 if fam == "forward" else 2
            work = sector_pairs_per_state(n // 2, na, nb, ijab) * 4 * amp_bytes * vecs * B
            peak = dev_pk["smem_gbs"]
            achieved, unit, bound = work / (ms / 1e3) / 1e9, "GB/s", "smem"
            basis = ("shared-memory bytes of the sector's active pairs: 2 loads + 2 stores "
                     "per pair, factor and vector")
            peak_kind = "derived: SMs x 32 banks x 4 B x max SM clock"
        hbm = sector_bytes(fam, info, amp_bytes, B)
        fs, fs_kind = full_space_work(fam, n, amp_bytes, ijab, info["n_groups"])
        fams[fam] = {
            "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "basis": basis, "peak_kind": peak_kind,
            "ms_per_step": ms, "launches_per_step": launches,
            "algorithmic_per_launch": work / max(1.0, launches),
            "avg_launch_ms": ms / max(1.0, launches),
            "hbm_sector": {"bytes_per_step": hbm, "achieved": hbm / (ms / 1e3) / 1e9,
                           "peak": pk["hbm_gbs"], "unit": "GB/s",
                           "frac": hbm / (ms / 1e3) / 1e9 / pk["hbm_gbs"],
                           "peak_kind": pk_kind,
                           "note": "compulsory sector bytes in HBM (psi, sigma and the "
                                   "hand-over between runs)"},
            "full_space_equivalent": {
                "work_per_step": fs * B, "unit": fs_kind + "/s",
                "rate": fs * B / (ms / 1e3),
                "note": "the same work counted over all 2^n amplitudes; the kernels skip the "
                        "amplitudes outside the electron sector, so this is no fraction of a "
                        "peak"}}
    dom = max(fams, key=lambda f: fams[f]["ms_per_step"])
    d = fams[dom]
    return {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
            "unit": d["unit"], "frac": d["frac"], "traffic": recorded_traffic(dom, workload),
            "basis": d["basis"], "peak_kind": d["peak_kind"],
            "sm_count": dev_pk["sm_count"], "sm_max_mhz": dev_pk["sm_max_mhz"],
            "families": fams}


def sector_pairs_per_state(n_orb, na, nb, ijab):
    """Active pairs of the electron sector over the excitation list: for
    each excitation the sector determinants with its occupied orbitals
    filled and its virtual orbitals empty."""
    from math import comb
    pairs = 0
    for row in np.asarray(ijab).reshape(-1, 4).tolist():
        qs = [q for q in row if q >= 0]
        ka = sum(1 for q in qs if q % 2 == 0) // 2
        kb = sum(1 for q in qs if q % 2 == 1) // 2
        pairs += comb(n_orb - 2 * ka, na - ka) * comb(n_orb - 2 * kb, nb - kb)
    return pairs


def sector_updates_per_state(n_orb, na, nb):
    """Connected group contributions per evaluation of one state on the
    (na, nb) sector: for every sector amplitude the diagonal, its same-spin
    singles and doubles and the mixed alpha-beta doubles."""
    from math import comb
    sa, sb = na * (n_orb - na), nb * (n_orb - nb)
    da = comb(na, 2) * comb(n_orb - na, 2)
    db = comb(nb, 2) * comb(n_orb - nb, 2)
    per_amp = 1 + sa + sb + da + db + sa * sb
    return per_amp * comb(n_orb, na) * comb(n_orb, nb)


def run_ours(args):
    import torch
    import paper_2402_17993_gb300 as uc

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = uc.FP32_STATE if args.precision == "fp32" else uc.FP64
    amp_bytes = 8 if prec == uc.FP32_STATE else 16
    w = synth.workload(args.workload)
    B = args.batch
    layout = uc.LAYOUT_SECTOR if args.layout == "sector" else uc.LAYOUT_FULL
    ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                          precision=prec, device=local, batch=B, layout=layout)
    K = ctx.K
    std, seed0 = (0.05, 1002) if args.workload == "18q" else (0.02, 1004)
    th_host = np.stack([synth.theta_normal(K, std, seed0 + b + 1000 * rank) for b in range(B)])
    theta = torch.tensor(th_host, device=dev, dtype=torch.float64)
    E = torch.empty(B, device=dev, dtype=torch.float64)
    G = torch.empty(B, K, device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        ctx.energy_grad_device(theta, E, G, stream)
    barrier()
    ctx.set_profiling(True)
    launches0 = ctx.info()["launches"]
    clocks = clock_sampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for s in range(args.steps):
        flush.fill_(s & 0xFF)  # evict L2 between timed steps (not timed)
        evs[s][0].record(stream)
        ctx.energy_grad_device(theta, E, G, stream)
        evs[s][1].record(stream)
    barrier()
    ck = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    prof = ctx.profile()
    ctx.set_profiling(False)
    launches = ctx.info()["launches"] - launches0
    total_ms = reduce_max(total_ms, world)
    value = whole_job_rate(B * args.steps, world, total_ms)

    # end to end through the C ABI with pinned host buffers
    th_pin = torch.tensor(th_host, dtype=torch.float64).pin_memory()
    E_pin = torch.empty(B, dtype=torch.float64).pin_memory()
    G_pin = torch.empty(B, K, dtype=torch.float64).pin_memory()
    # each step from host buffers to host buffers, timed on the host (the call
    # returns once the results are in E_pin and G_pin), with L2 evicted and the
    # device idle before it as in the device-timed loop (not timed)
    barrier()
    e2e_s = 0.0
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.energy_grad_ptr(B, th_pin.data_ptr(), E_pin.data_ptr(), G_pin.data_ptr(), False, stream)
        e2e_s += time.perf_counter() - t0
    barrier()
    e2e_s = reduce_max(e2e_s * 1e3, world) * 1e-3
    e2e = {"value": world * B * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": B * K * 8, "d2h_bytes_per_step": B * 8 + B * K * 8,
           "l2": "evicted before each step (not timed)"}

    info = ctx.info()
    ijab = uc.build_uccsd_list(w["n_orb"], w["n_alpha"], w["n_beta"])
    workload = f"{args.workload}_b{B}_{args.precision}"
    dev_pk = device_peaks(torch.cuda.get_device_properties(dev).multi_processor_count,
                          ck.get("sm_max_mhz") or 2070.0)
    roof = roofline(prof, B, info, amp_bytes, ijab, prec == uc.FP32_STATE, workload, dev_pk)

    line = {
        "metric": METRIC if args.workload == "18q" else METRIC_26Q, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == uc.FP32_STATE else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "18q" else WORKLOAD_26Q,
                   "state": ("real amplitudes as FP32 hi + lo (8 bytes), FP64 reductions"
                             if prec else "complex128"),
                   "layout": args.layout + (" (2^n vector per slot)" if args.layout == "full"
                                            else " (electron-sector array per slot)"),
                   "l2": "flushed between timed steps (256 MB write)",
                   "fwd_runs": info["n_fwd_runs"], "adj_runs": info["n_adj_runs"],
                   "groups": info["n_groups"], "terms": info["n_terms"]},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": ck,
    }
    if args.workload != "18q":
        # the oracle takes about 15 minutes per 26-qubit evaluation on the host
        # cores, and the other measurements are 18-qubit ones
        args.no_cpu_baseline = args.no_small = args.no_scaleup = args.no_serving = True
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        thetas = [th_host[b] for b in range(B)]
        rate, dt, cores = oracle_rate(w, thetas, 12)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"12 of the 64 theta vectors ({dt:.1f} s, sector-restricted "
                                          "FP64 oracle, OpenMP)"}
        try:
            line["cpu_baseline"]["single_core"] = {
                "value": oracle_rate_single_thread(), "unit": UNIT, "cores": 1,
                "sample": "1 theta vector (seed 1002), OMP_NUM_THREADS=1"}
        except Exception as exc:  # a missing single-core figure must not cost the bench line
            line["cpu_baseline"]["single_core"] = {"unavailable": str(exc)[:200]}
    if rank == 0 and not args.no_layout_compare and args.layout == "full":
        line["sector_layout"] = layout_compare(uc, local, w, prec, B, th_host, args, flush)
    if rank == 0 and not args.no_fp64_compare and prec == uc.FP32_STATE:
        line["fp64_b1"] = fp64_compare(uc, local, w, th_host, E, G, args.layout)
    if rank == 0 and not args.no_small:
        line["small"] = small_workloads(uc, local)
    if rank == 0 and not args.no_scaleup:
        line["scaleup"] = scaleup_26q(uc, local, dev_pk)
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_stream(uc, local, args.serving_requests,
                                         args.serving_fp64_requests)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def layout_compare(uc, device, w, prec, B, th_host, args, flush):
    """The same timed loop with the electron-sector state layout (bitwise the
    same results; a comparison beside the headline, which times the full
    2^n layout)."""
    import torch
    ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                          precision=prec, device=device, batch=B, layout=uc.LAYOUT_SECTOR)
    theta = torch.tensor(th_host, device="cuda", dtype=torch.float64)
    E = torch.empty(B, device="cuda", dtype=torch.float64)
    G = torch.empty(B, ctx.K, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.energy_grad_device(theta, E, G, stream)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        evs[s][0].record(stream)
        ctx.energy_grad_device(theta, E, G, stream)
        evs[s][1].record(stream)
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in evs)
    prof = ctx.profile()
    out = {"value": B * args.steps / (total / 1e3), "unit": UNIT,
           "ms_per_step": total / args.steps,
           "family_ms": {f: prof["ms"][f] / max(1, prof["calls"]) for f in prof["ms"]},
           "device_bytes": ctx.info()["device_bytes"]}
    ctx.close()
    return out


def fp64_compare(uc, device, w, th_host, E32, G32, layout_name):
    """The same 18q workload in the FP64 form, one state per call: its
    evaluation rate, and the error of the batched FP32-state evaluations of
    the timed loop against FP64 evaluations at the same 64 theta vectors (the
    FP64 path itself matches the oracle to 1e-10 in the parity tests)."""
    import torch
    layout = uc.LAYOUT_SECTOR if layout_name == "sector" else uc.LAYOUT_FULL
    ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                          precision=uc.FP64, device=device, batch=1, layout=layout)
    K = ctx.K
    th = torch.tensor(th_host, device="cuda", dtype=torch.float64)
    E = torch.empty(1, device="cuda", dtype=torch.float64)
    G = torch.empty(1, K, device="cuda", dtype=torch.float64)
    E64, G64 = [], []
    for b in range(th.shape[0]):
        ctx.energy_grad_device(th[b:b + 1], E, G)
        E64.append(float(E[0].item()))
        G64.append(G[0].cpu().numpy().copy())
    steps = 16
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for s_ in range(steps):
        ctx.energy_grad_device(th[s_ % th.shape[0]:s_ % th.shape[0] + 1], E, G)
    z.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / steps
    e32 = E32.cpu().numpy()
    g32 = G32.cpu().numpy()
    del ctx
    torch.cuda.empty_cache()
    g64 = np.stack(G64)
    return {"evals_per_s": 1e3 / ms, "ms_per_eval": ms, "batch": 1,
            "fp32_state_vs_fp64": {
                "max_abs_dE": float(np.max(np.abs(e32 - np.array(E64)))),
                "max_abs_dgrad": float(np.max(np.abs(g32 - g64))),
                "max_abs_g": float(np.max(np.abs(g64))),
                "evals_compared": int(th.shape[0])}}


def small_workloads(uc, device):
    """The two small workloads, each in FP64 and in the FP32-state form.

    8 qubits (4 electrons, seed 0): one energy + gradient at theta0 ~
    U(-0.1, 0.1) and the 16-point sweep theta0 + phi_s e_k along the first
    double (phi_s = -pi + 2 pi s / 16), against the oracle's stored values;
    along one amplitude the energy is a trigonometric polynomial of degree
    2, so the sweep's DFT content above frequency 2 measures rounding only.

    12 qubits (6 electrons, seed 1): VQE by L-BFGS-B with the adjoint
    gradient from theta = 0 to a gradient 2-norm below 1e-6 (both
    precisions; the 2-norm reached is reported), with the
    iterations, evaluations, rate and final energy against the stored FCI
    energy, and the FP32-state energy at the FP64 optimum."""
    import time as _t

    from paper_2402_17993_gb300 import vqe
    gdir = os.path.join(ROOT, "tests", "golden")
    out = {}
    g8 = json.load(open(os.path.join(gdir, "golden_8q.json")))
    w = synth.workload("8q")
    K8 = len(uc.build_uccsd_list(w["n_orb"], w["n_alpha"], w["n_beta"]))
    th0 = synth.theta_uniform(K8, -0.1, 0.1, 1000)
    k = g8["sweep_k"]
    sweep = np.tile(th0, (16, 1))
    sweep[:, k] += -np.pi + 2 * np.pi * np.arange(16) / 16
    for name, prec in (("fp64", uc.FP64), ("fp32_state", uc.FP32_STATE)):
        ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                              precision=prec, device=device)
        ctx.energy_grad(np.zeros(ctx.K))  # first launches load the kernels: not timed
        E, g = ctx.energy_grad(th0)
        Es = np.array([ctx.energy(t) for t in sweep])
        t0 = _t.perf_counter()
        for t in sweep:
            ctx.energy_grad(t)
        dt = (_t.perf_counter() - t0) / 16
        F = np.abs(np.fft.rfft(Es)) / 16
        out[f"8q_{name}"] = {
            "abs_dE_vs_oracle": abs(E - g8["E"]),
            "max_abs_dgrad_vs_oracle": float(np.max(np.abs(g - np.array(g8["grad"])))),
            "sweep_max_abs_dE_vs_oracle": float(np.max(np.abs(Es - np.array(g8["sweep_E"])))),
            "sweep_dft_above_2": float(np.max(F[3:])),
            "ms_per_eval_host_call": 1e3 * dt}
        ctx.close()
    g12 = json.load(open(os.path.join(gdir, "golden_12q.json")))
    w = synth.workload("12q")
    res = {}
    for name, prec, gtol in (("fp64", uc.FP64, 1e-6), ("fp32_state", uc.FP32_STATE, 1e-6)):
        ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                              precision=prec, device=device)
        ctx.energy_grad(np.zeros(ctx.K))  # first launches load the kernels: not timed
        t0 = _t.perf_counter()
        E, theta, n_eval, gnorm = vqe.minimize(ctx, gtol=gtol)
        dt = _t.perf_counter() - t0
        res[name] = (ctx, theta, E)
        out[f"12q_vqe_{name}"] = {
            "gtol": gtol, "evals": n_eval, "grad_norm": gnorm, "E": E,
            "E_minus_fci": E - g12["E_fci"], "E_hf": g12["E_hf"], "E_fci": g12["E_fci"],
            "evals_per_s_host_loop": n_eval / dt, "seconds": dt}
    ctx64, th64, E64 = res["fp64"]
    ctx32 = res["fp32_state"][0]
    out["12q_vqe_fp32_state"]["abs_dE_at_fp64_optimum"] = abs(ctx32.energy(th64) - E64)
    out["12q_vqe_fp32_state"]["abs_dE_converged_vs_fp64"] = abs(res["fp32_state"][2] - E64)
    ctx64.close()
    ctx32.close()
    return out


def scaleup_26q(uc, device, dev_pk):
    import torch
    w = synth.workload("26q")
    gold_path = os.path.join(ROOT, "tests", "golden", "golden_26q.json")
    gold = json.load(open(gold_path)) if os.path.exists(gold_path) else None
    out = {}
    for name, prec, layout in (("fp32", uc.FP32_STATE, uc.LAYOUT_FULL),
                               ("fp64", uc.FP64, uc.LAYOUT_FULL),
                               ("fp32_sector_layout", uc.FP32_STATE, uc.LAYOUT_SECTOR),
                               ("fp64_sector_layout", uc.FP64, uc.LAYOUT_SECTOR)):
        ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"],
                              w["n_beta"], precision=prec, device=device, layout=layout)
        th = torch.tensor(synth.theta_normal(ctx.K, 0.02, 1004), device="cuda",
                          dtype=torch.float64).unsqueeze(0)
        E = torch.empty(1, device="cuda", dtype=torch.float64)
        G = torch.empty(1, ctx.K, device="cuda", dtype=torch.float64)
        ctx.energy_grad_device(th, E, G)
        torch.cuda.synchronize()
        ctx.set_profiling(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 2
        a.record()
        for _ in range(steps):
            ctx.energy_grad_device(th, E, G)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        prof = ctx.profile()
        inf = ctx.info()
        err = {}
        if gold is not None:
            err = {"abs_dE_vs_oracle": abs(float(E[0].item()) - gold["E"]),
                   "max_abs_dgrad_vs_oracle": float(np.max(np.abs(G[0].cpu().numpy()
                                                                  - np.array(gold["grad"]))))}
        ijab = uc.build_uccsd_list(w["n_orb"], w["n_alpha"], w["n_beta"])
        amp = 8 if prec == uc.FP32_STATE else 16
        fams = roofline(prof, 1, inf, amp, ijab, prec == uc.FP32_STATE,
                        f"26q_b1_{name}", dev_pk)["families"]
        out[name] = {"evals_per_s": 1e3 / ms, "ms_per_eval": ms, "E": float(E[0].item()), **err,
                     "family_ms": {f: prof["ms"][f] / max(1, prof["calls"]) for f in prof["ms"]},
                     "fwd_runs": inf["n_fwd_runs"], "adj_runs": inf["n_adj_runs"],
                     "families": {f: {k: v[k] for k in ("bound", "achieved", "peak", "unit",
                                                          "frac", "ms_per_step",
                                                          "launches_per_step", "hbm_sector")}
                                  for f, v in fams.items()}}
        del ctx
        torch.cuda.empty_cache()
    return out


def serving_stream(uc, device, n_req, n_req_fp64):
    """FMO fragment stream (60% monomers at 8-12 qubits, 40% dimers at 16-18
    qubits, 40 fixed-step L-BFGS evaluations per solve): capacity of the
    batched FP32 server (closed loop), latency percentiles at 0.5x, 0.8x and
    1.2x that capacity with Poisson arrivals (seed 7), and the
    one-request-at-a-time FP64 form on the same requests, with the final
    energy of every fragment compared between the two forms."""
    from paper_2402_17993_gb300.serving import FragmentServer, Request, capacity_rate
    frags = synth.stream_fragments(n_req, 7)
    reqs = [Request(d["r"], d["t_unit"], d["n_orb"], d["n_alpha"], d["n_beta"], d["h"], d["eri"],
                    d["e_core"]) for d in frags]
    n64 = n_req if n_req_fp64 is None else min(n_req_fp64, n_req)
    out = {}
    srv = FragmentServer(precision=uc.FP32_STATE, device=device, max_active=64)
    srv.run(reqs[:64])  # warm the context pool and graph paths
    res32, cap = srv.run(reqs, keep_theta=True)
    rate = capacity_rate(cap)
    out["batched_fp32"] = {"closed_loop": cap}
    for f in (0.5, 0.8, 1.2):
        _, op = srv.run(reqs, rate=f * rate)
        out["batched_fp32"][f"open_loop_{f}x"] = dict(op, rate_req_per_s=f * rate)
    # the same arrivals with the next 8 requests prepared ahead of their
    # arrival, each solve waiting behind a device gate that the serving
    # thread releases at the arrival (instead of being set up and launched
    # then)
    srv.lookahead = 8
    for f in (0.5, 0.8):
        _, op = srv.run(reqs, rate=f * rate)
        out["batched_fp32"][f"open_loop_{f}x_gated_lookahead8"] = dict(op, rate_req_per_s=f * rate)
    srv.lookahead = 0
    srv.close()
    one = FragmentServer(precision=uc.FP64, device=device, max_active=1, n_streams=1,
                         use_graphs=False)
    res64, st1 = one.run(reqs[:n64])
    one.close()
    e32 = {r.r: r.energy for r in res32}
    dE = np.array([abs(e32[r.r] - r.energy) for r in res64])
    out["one_at_a_time_fp64"] = dict(st1, note=f"the first {n64} requests of the same stream "
                                               f"(closed loop)")
    # evaluation precision: both forms at the same amplitudes (each
    # fragment's final theta of the batched run)
    by_r = {q.r: q for q in reqs}
    ctxs = {}
    same = []
    for r in res32[:n64]:
        q = by_r[r.r]
        key = (q.n_orb, q.n_alpha, q.n_beta)
        if key not in ctxs:
            ctxs[key] = [uc.Context(device, p) for p in (uc.FP32_STATE, uc.FP64)]
        es = []
        for c in ctxs[key]:
            c.set_hamiltonian(q.n_orb, q.h, q.eri, q.e_core).set_reference(q.n_alpha, q.n_beta)
            c.set_excitations(uc.build_uccsd_list(q.n_orb, q.n_alpha, q.n_beta))
            es.append(c.energy(r.theta))
        same.append(abs(es[0] - es[1]))
    for cs in ctxs.values():
        for c in cs:
            c.close()
    same = np.array(same)
    out["fp32_batched_vs_fp64_one_at_a_time"] = {
        "fragments": int(len(dE)),
        "same_theta_max_abs_dE": float(same.max()),
        "same_theta_median_abs_dE": float(np.median(same)),
        "final_max_abs_dE": float(dE.max()), "final_median_abs_dE": float(np.median(dE)),
        "final_within_1e-5": int(np.sum(dE <= 1e-5)),
        "note": "same_theta: both precisions evaluated at each fragment's final amplitudes "
                "(the evaluation error); final: the last energy of each form's own 40-step "
                "fixed-step L-BFGS run (device optimiser for the batched form, host optimiser "
                "for the other), where the two trajectories may separate"}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
