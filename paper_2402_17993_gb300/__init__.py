"""GB300 (sm_103a) VQE-UCCSD state-vector library: Python binding.

Thin ctypes marshalling over the C ABI declared in ``include/uccsd.h``
(Trotterised UCCSD energy and adjoint gradient of arXiv:2402.17993,
Eqs. 2-6).  Every step of the computation runs in the CUDA library; this
module only moves arguments.  PyTorch is used for device tensors and
streams.  If the compiled library is missing, importing a function that
needs it raises immediately: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libuccsd_gb300.so")

FP64 = 0
FP32_STATE = 1
LAYOUT_FULL = 0
LAYOUT_SECTOR = 1
LAYOUT_SCBK = 2

STATUS = {0: "ok", 1: "invalid argument", 2: "device out of memory", 3: "CUDA error",
          4: "invalid call order or failed context", 5: "device wait timed out",
          6: "HBM budget exceeded"}

# Symbols of include/uccsd.h (checked by the CPU test suite).
EXPORTS = [
    "uccsd_create", "uccsd_destroy", "uccsd_last_error", "uccsd_status_string",
    "uccsd_set_hamiltonian", "uccsd_set_reference", "uccsd_build_uccsd_list",
    "uccsd_set_excitations", "uccsd_set_batch", "uccsd_energy", "uccsd_energy_grad",
    "uccsd_energy_grad_batch", "uccsd_get_state", "uccsd_info", "uccsd_hamiltonian_stats",
    "uccsd_pauli_terms", "uccsd_set_profiling", "uccsd_get_profile", "uccsd_expectation_noalloc",
    "uccsd_capture", "uccsd_replay", "uccsd_mp1_amplitudes", "uccsd_magnitude_order",
    "uccsd_trotter_extrapolate", "uccsd_energy_trotter_free", "uccsd_energy_grad_trotter_free",
    "uccsd_set_layout", "uccsd_pauli_terms_scbk", "uccsd_opt_init", "uccsd_opt_step",
    "uccsd_opt_history", "uccsd_set_setup_stream", "uccsd_capture_vqe_step",
    "uccsd_energy_grad_batched", "uccsd_plan_pairs", "uccsd_gate_enqueue", "uccsd_gate_status",
    "uccsd_happly_mixed_order", "uccsd_stream_mark", "uccsd_mark_done", "uccsd_zero_async",
    "uccsd_plan_entry_map",
]

FAMILIES = ["cs", "forward", "happly", "adjoint", "reduce"]


class UCCSDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Info(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("n_orb", ctypes.c_int), ("n_alpha", ctypes.c_int),
                ("n_beta", ctypes.c_int), ("K", ctypes.c_int), ("n_ops", ctypes.c_int),
                ("n_groups", ctypes.c_int), ("n_terms", ctypes.c_int),
                ("n_fwd_runs", ctypes.c_int), ("n_adj_runs", ctypes.c_int),
                ("batch", ctypes.c_int), ("precision", ctypes.c_int), ("layout", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("launches", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 5), ("launches", ctypes.c_uint64 * 5),
                ("calls", ctypes.c_uint64)]


_lib = None


def lib():
    """Load the compiled library; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"UCCSD CUDA library not built ({LIB_PATH}); "
                               "run `python -m paper_2402_17993_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        f64p = ctypes.POINTER(ctypes.c_double)
        L.uccsd_create.argtypes = [ctypes.POINTER(vp), ip, ip, ctypes.c_size_t]
        L.uccsd_destroy.argtypes = [vp]
        L.uccsd_destroy.restype = None
        L.uccsd_last_error.argtypes = [vp]
        L.uccsd_last_error.restype = ctypes.c_char_p
        L.uccsd_status_string.argtypes = [ip]
        L.uccsd_status_string.restype = ctypes.c_char_p
        L.uccsd_set_hamiltonian.argtypes = [vp, ip, f64p, f64p, ctypes.c_double]
        L.uccsd_set_reference.argtypes = [vp, ip, ip]
        L.uccsd_set_layout.argtypes = [vp, ip]
        L.uccsd_set_setup_stream.argtypes = [vp, vp]
        L.uccsd_build_uccsd_list.argtypes = [ip, ip, ip, i32p, ip, ctypes.POINTER(ctypes.c_int)]
        L.uccsd_set_excitations.argtypes = [vp, ip, i32p, ip, ip]
        L.uccsd_set_batch.argtypes = [vp, ip]
        L.uccsd_energy.argtypes = [vp, dp, ip, dp, vp]
        L.uccsd_energy_grad.argtypes = [vp, dp, ip, dp, dp, vp]
        L.uccsd_energy_grad_batch.argtypes = [vp, ip, dp, ip, dp, dp, vp]
        L.uccsd_get_state.argtypes = [vp, ip, f64p, ctypes.c_size_t]
        L.uccsd_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.uccsd_hamiltonian_stats.argtypes = [ip, f64p, f64p, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]
        L.uccsd_expectation_noalloc.argtypes = [vp, vp, vp, vp]
        L.uccsd_capture.argtypes = [vp, ip, dp, dp, dp, vp]
        L.uccsd_replay.argtypes = [vp, vp]
        L.uccsd_capture_vqe_step.argtypes = [vp, dp, dp, dp, vp]
        vpp = ctypes.POINTER(vp)
        L.uccsd_energy_grad_batched.argtypes = [vpp, ip, vpp, dp, vpp, vp]
        L.uccsd_set_profiling.argtypes = [vp, ip]
        L.uccsd_get_profile.argtypes = [vp, ctypes.POINTER(Profile)]
        L.uccsd_pauli_terms.argtypes = [ip, f64p, f64p, ctypes.c_double, u32p, u32p, f64p, ip,
                                        ctypes.POINTER(ctypes.c_int)]
        L.uccsd_mp1_amplitudes.argtypes = [vp, f64p, vp]
        L.uccsd_opt_init.argtypes = [vp, ip, ctypes.c_double, ctypes.c_double, ip]
        L.uccsd_opt_step.argtypes = [vp, dp, dp, dp, vp]
        L.uccsd_opt_history.argtypes = [vp, f64p, ip, ctypes.POINTER(ctypes.c_int)]
        L.uccsd_pauli_terms_scbk.argtypes = [ip, f64p, f64p, ctypes.c_double, ip, ip, u32p, u32p,
                                             f64p, ip, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]
        L.uccsd_energy_trotter_free.argtypes = [vp, dp, ip, dp, vp]
        L.uccsd_energy_grad_trotter_free.argtypes = [vp, dp, ip, dp, dp, vp]
        L.uccsd_magnitude_order.argtypes = [ip, i32p, f64p, i32p, i32p]
        L.uccsd_trotter_extrapolate.argtypes = [ip, ctypes.POINTER(ctypes.c_int), f64p, f64p]
        L.uccsd_plan_pairs.argtypes = [ip, ip, ip, i32p, ip, ip, ip, i32p, ip,
                                       ctypes.POINTER(ctypes.c_int)]
        L.uccsd_happly_mixed_order.argtypes = [ip, ip, i32p, ip, ctypes.POINTER(ctypes.c_int)]
        L.uccsd_plan_entry_map.argtypes = [ip, ip, ip, i32p, ip, ip, ip, i32p, ip,
                                           ctypes.POINTER(ctypes.c_int)]
        L.uccsd_stream_mark.argtypes = [vp, vp]
        L.uccsd_mark_done.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.uccsd_zero_async.argtypes = [vp, vp, ctypes.c_size_t, vp]
        L.uccsd_gate_enqueue.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint64, vp]
        L.uccsd_gate_status.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int)]
        _lib = L
    return _lib


def _f64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Host-only entry points
# ---------------------------------------------------------------------------
def build_uccsd_list(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    L = lib()
    n = ctypes.c_int(0)
    st = L.uccsd_build_uccsd_list(n_orb, n_alpha, n_beta, None, 0, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "build_uccsd_list")
    out = np.zeros((n.value, 4), dtype=np.int32)
    st = L.uccsd_build_uccsd_list(n_orb, n_alpha, n_beta, _i32p(out), n.value, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "build_uccsd_list")
    return out


def plan_pairs(n_orb, n_alpha, n_beta, ijab, amp_bytes=8, nvec=1):
    """Host-only: the sweep plan's precomputed pair lists in determinant
    space, one row (factor, first, second, sign, entry, partner entry,
    index) per pair (uccsd_plan_pairs)."""
    ijab = np.ascontiguousarray(ijab, dtype=np.int32).reshape(-1, 4)
    n = ctypes.c_int(0)
    st = lib().uccsd_plan_pairs(n_orb, n_alpha, n_beta, _i32p(ijab), ijab.shape[0], amp_bytes,
                                nvec, None, 0, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "plan_pairs")
    out = np.zeros((n.value, 7), dtype=np.int32)
    st = lib().uccsd_plan_pairs(n_orb, n_alpha, n_beta, _i32p(ijab), ijab.shape[0], amp_bytes,
                                nvec, _i32p(out), n.value, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "plan_pairs")
    return out


def plan_entry_map(n_orb, n_alpha, n_beta, ijab, amp_bytes=8, nvec=1):
    """Host-only: the sweep plan's entry maps, one row (run, tile, entry,
    sector index, determinant) per tile entry (uccsd_plan_entry_map)."""
    ijab = np.ascontiguousarray(ijab, dtype=np.int32).reshape(-1, 4)
    n = ctypes.c_int(0)
    st = lib().uccsd_plan_entry_map(n_orb, n_alpha, n_beta, _i32p(ijab), ijab.shape[0], amp_bytes,
                                    nvec, None, 0, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "plan_entry_map")
    out = np.zeros((n.value, 5), dtype=np.int32)
    st = lib().uccsd_plan_entry_map(n_orb, n_alpha, n_beta, _i32p(ijab), ijab.shape[0], amp_bytes,
                                    nvec, _i32p(out), n.value, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "plan_entry_map")
    return out


def happly_mixed_order(n_orb, n_beta):
    """Host-only: the slot order of every column's beta singles in the FP32
    H-apply's mixed groups, shape (n_singles, C(n_orb, n_beta)); entry
    [t, column] = the natural index of the single taken at slot t
    (uccsd_happly_mixed_order)."""
    n = ctypes.c_int(0)
    st = lib().uccsd_happly_mixed_order(n_orb, n_beta, None, 0, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "happly_mixed_order")
    out = np.zeros(n.value, dtype=np.int32)
    st = lib().uccsd_happly_mixed_order(n_orb, n_beta, _i32p(out), n.value, ctypes.byref(n))
    if st:
        raise UCCSDError(st, "happly_mixed_order")
    from math import comb
    return out.reshape(n_beta * (n_orb - n_beta), comb(n_orb, n_beta))


def hamiltonian_stats(n_orb, h, eri, e_core=0.0):
    g, t = ctypes.c_int(0), ctypes.c_int(0)
    h, eri = _c64(h), _c64(eri)
    st = lib().uccsd_hamiltonian_stats(n_orb, _f64p(h), _f64p(eri), float(e_core),
                                       ctypes.byref(g), ctypes.byref(t))
    if st:
        raise UCCSDError(st, "hamiltonian_stats")
    return g.value, t.value


def pauli_terms(n_orb, h, eri, e_core=0.0):
    """Compiled Jordan-Wigner terms: (xmask, zmask, coef) with
    H = sum coef X^xmask Z^zmask."""
    L = lib()
    h, eri = _c64(h), _c64(eri)
    n = ctypes.c_int(0)
    st = L.uccsd_pauli_terms(n_orb, _f64p(h), _f64p(eri), float(e_core), None, None, None, 0,
                             ctypes.byref(n))
    if st:
        raise UCCSDError(st, "pauli_terms")
    x = np.zeros(n.value, dtype=np.uint32)
    z = np.zeros(n.value, dtype=np.uint32)
    c = np.zeros(n.value, dtype=np.float64)
    st = L.uccsd_pauli_terms(n_orb, _f64p(h), _f64p(eri), float(e_core),
                             x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                             z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _f64p(c), n.value,
                             ctypes.byref(n))
    if st:
        raise UCCSDError(st, "pauli_terms")
    return x, z, c


def pauli_terms_scbk(n_orb, h, eri, e_core, n_alpha, n_beta):
    """Symmetry-conserving Bravyi-Kitaev terms with two qubits tapered:
    (xmask, zmask, coef, n_qubits)."""
    L = lib()
    h, eri = _c64(h), _c64(eri)
    n, nq = ctypes.c_int(0), ctypes.c_int(0)
    st = L.uccsd_pauli_terms_scbk(n_orb, _f64p(h), _f64p(eri), float(e_core), n_alpha, n_beta,
                                  None, None, None, 0, ctypes.byref(n), ctypes.byref(nq))
    if st:
        raise UCCSDError(st, "pauli_terms_scbk")
    x = np.zeros(n.value, dtype=np.uint32)
    z = np.zeros(n.value, dtype=np.uint32)
    c = np.zeros(n.value, dtype=np.float64)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    st = L.uccsd_pauli_terms_scbk(n_orb, _f64p(h), _f64p(eri), float(e_core), n_alpha, n_beta,
                                  x.ctypes.data_as(u32), z.ctypes.data_as(u32), _f64p(c), n.value,
                                  ctypes.byref(n), ctypes.byref(nq))
    if st:
        raise UCCSDError(st, "pauli_terms_scbk")
    return x, z, c, nq.value


def magnitude_order(ijab, t):
    """Rows of ijab by decreasing |t| (stable); returns (rows, perm) with
    rows = ijab[perm]."""
    ijab = np.ascontiguousarray(ijab, dtype=np.int32).reshape(-1, 4)
    t = _c64(t).reshape(ijab.shape[0])
    out = np.zeros_like(ijab)
    perm = np.zeros(ijab.shape[0], dtype=np.int32)
    st = lib().uccsd_magnitude_order(ijab.shape[0], _i32p(ijab), _f64p(t), _i32p(out), _i32p(perm))
    if st:
        raise UCCSDError(st, "magnitude_order")
    return out, perm


def trotter_extrapolate(Ms, Es):
    """Fit E(M) = alpha (1/M)^beta + gamma; returns (alpha, beta, gamma)."""
    M = np.ascontiguousarray(Ms, dtype=np.int32)
    E = _c64(Es).reshape(M.shape[0])
    out = np.zeros(3)
    st = lib().uccsd_trotter_extrapolate(M.shape[0], M.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                         _f64p(E), _f64p(out))
    if st:
        raise UCCSDError(st, "trotter_extrapolate")
    return float(out[0]), float(out[1]), float(out[2])


# ---------------------------------------------------------------------------
# Context
# ---------------------------------------------------------------------------
def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One fragment (Hamiltonian + reference + excitation list) on one GPU."""

    def __init__(self, device: int = 0, precision: int = FP64, hbm_budget_bytes: int = 0):
        self._L = lib()
        self._c = ctypes.c_void_p(None)
        st = self._L.uccsd_create(ctypes.byref(self._c), device, precision, hbm_budget_bytes)
        if st:
            raise UCCSDError(st, "uccsd_create")
        self.device = device
        self.precision = precision
        self.K = 0
        self.n_qubits = 0

    def _check(self, st, what):
        if st:
            msg = self._L.uccsd_last_error(self._c).decode()
            raise UCCSDError(st, f"{what}: {msg}")

    def close(self):
        if self._c:
            self._L.uccsd_destroy(self._c)
            self._c = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_hamiltonian(self, n_orb, h, eri, e_core=0.0):
        h, eri = _c64(h), _c64(eri)
        self._check(self._L.uccsd_set_hamiltonian(self._c, n_orb, _f64p(h), _f64p(eri),
                                                  float(e_core)), "set_hamiltonian")
        self.n_qubits = 2 * n_orb
        return self

    def set_setup_stream(self, stream=None):
        """Enqueue later set-up transfers on `stream` without host waits
        (None: the context's own stream, waited on by each call)."""
        ptr = ctypes.c_void_p(None) if stream is None else _stream_ptr(stream)
        self._check(self._L.uccsd_set_setup_stream(self._c, ptr), "set_setup_stream")
        return self

    def set_layout(self, layout):
        self._check(self._L.uccsd_set_layout(self._c, layout), "set_layout")
        return self

    def set_reference(self, n_alpha, n_beta):
        self._check(self._L.uccsd_set_reference(self._c, n_alpha, n_beta), "set_reference")
        return self

    def set_excitations(self, ijab, trotter_order=1, n_slices=1):
        ijab = np.ascontiguousarray(ijab, dtype=np.int32).reshape(-1, 4)
        self._check(self._L.uccsd_set_excitations(self._c, ijab.shape[0], _i32p(ijab),
                                                  trotter_order, n_slices), "set_excitations")
        self.K = ijab.shape[0]
        return self

    def set_batch(self, B):
        self._check(self._L.uccsd_set_batch(self._c, B), "set_batch")
        return self

    # -- host-buffer calls (synchronising) --
    def energy(self, theta, stream=None):
        th = _c64(theta).reshape(self.K)
        E = np.zeros(1)
        self._check(self._L.uccsd_energy(self._c, th.ctypes.data, 0, E.ctypes.data,
                                         _stream_ptr(stream)), "energy")
        return float(E[0])

    def energy_grad(self, theta, stream=None):
        th = _c64(theta).reshape(self.K)
        E = np.zeros(1)
        g = np.zeros(max(self.K, 1))
        self._check(self._L.uccsd_energy_grad(self._c, th.ctypes.data, 0, E.ctypes.data,
                                              g.ctypes.data, _stream_ptr(stream)), "energy_grad")
        return float(E[0]), g[:self.K].copy()

    def energy_grad_batch(self, theta, grad=True, stream=None):
        th = _c64(theta).reshape(-1, self.K)
        B = th.shape[0]
        E = np.zeros(B)
        g = np.zeros((B, max(self.K, 1)))
        self._check(self._L.uccsd_energy_grad_batch(self._c, B, th.ctypes.data, 0, E.ctypes.data,
                                                    g.ctypes.data if grad else None,
                                                    _stream_ptr(stream)), "energy_grad_batch")
        return E, (g[:, :self.K].copy() if grad else None)

    # -- device-tensor calls (asynchronous on the stream) --
    def energy_grad_device(self, theta, E, grad, stream=None):
        """theta: CUDA float64 tensor (B, K) or (K,); E: (B,); grad: (B, K) or None."""
        B = 1 if theta.dim() == 1 else theta.shape[0]
        assert theta.is_cuda and theta.dtype.is_floating_point and theta.is_contiguous()
        gp = None if grad is None else grad.data_ptr()
        self._check(self._L.uccsd_energy_grad_batch(self._c, B, theta.data_ptr(), 1, E.data_ptr(),
                                                    gp, _stream_ptr(stream)),
                    "energy_grad_batch(device)")

    def capture(self, theta, E, grad, stream):
        """Capture one evaluation reading the CUDA tensor theta (B, K) into a
        graph writing E (B,) and grad (B, K) or None; replay() reruns it."""
        B = 1 if theta.dim() == 1 else theta.shape[0]
        gp = None if grad is None else grad.data_ptr()
        self._check(self._L.uccsd_capture(self._c, B, theta.data_ptr(), E.data_ptr(), gp,
                                          _stream_ptr(stream)), "capture")

    def capture_vqe_step(self, theta, E, grad, stream):
        """Capture evaluation + device optimiser step on the CUDA tensors
        theta (K,), E (1,), grad (K,); replay() then runs one VQE iteration."""
        self._check(self._L.uccsd_capture_vqe_step(self._c, theta.data_ptr(), E.data_ptr(),
                                                   grad.data_ptr(), _stream_ptr(stream)),
                    "capture_vqe_step")

    def replay(self, stream):
        self._check(self._L.uccsd_replay(self._c, _stream_ptr(stream)), "replay")

    def state(self, slot=0):
        """The state vector of `slot`: 2^n amplitudes, or the 2^(n-2) of the
        tapered encoding in LAYOUT_SCBK."""
        n = self.n_qubits - (2 if self.info()["layout"] == LAYOUT_SCBK else 0)
        N = 1 << n
        out = np.zeros(2 * N)
        self._check(self._L.uccsd_get_state(self._c, slot, _f64p(out), out.size), "get_state")
        return out.view(np.complex128)

    def set_profiling(self, on=True):
        self._check(self._L.uccsd_set_profiling(self._c, 1 if on else 0), "set_profiling")

    def profile(self):
        p = Profile()
        self._check(self._L.uccsd_get_profile(self._c, ctypes.byref(p)), "get_profile")
        return {"ms": dict(zip(FAMILIES, list(p.ms))),
                "launches": dict(zip(FAMILIES, list(p.launches))), "calls": p.calls}

    def energy_grad_ptr(self, B, theta_ptr, E_ptr, grad_ptr, on_device, stream=None):
        """Raw-pointer call (host pinned or device buffers)."""
        self._check(self._L.uccsd_energy_grad_batch(self._c, B, theta_ptr, 1 if on_device else 0,
                                                    E_ptr, grad_ptr, _stream_ptr(stream)),
                    "energy_grad_batch(ptr)")

    def energy_trotter_free(self, theta, stream=None):
        """E of exp(sum_k theta_k G_k)|HF> (no Trotterisation)."""
        th = _c64(theta).reshape(self.K)
        E = np.zeros(1)
        self._check(self._L.uccsd_energy_trotter_free(self._c, th.ctypes.data, 0, E.ctypes.data,
                                                      _stream_ptr(stream)), "energy_trotter_free")
        return float(E[0])

    def energy_grad_trotter_free(self, theta, stream=None):
        """E and dE/dtheta of exp(sum_k theta_k G_k)|HF>."""
        th = _c64(theta).reshape(self.K)
        E = np.zeros(1)
        g = np.zeros(max(self.K, 1))
        self._check(self._L.uccsd_energy_grad_trotter_free(self._c, th.ctypes.data, 0,
                                                           E.ctypes.data, g.ctypes.data,
                                                           _stream_ptr(stream)),
                    "energy_grad_trotter_free")
        return float(E[0]), g[:self.K].copy()

    def opt_init(self, memory=10, max_step=0.2, first_scale=0.1, max_steps=40):
        """Device fixed-step L-BFGS state (see uccsd_opt_init)."""
        self._check(self._L.uccsd_opt_init(self._c, memory, max_step, first_scale, max_steps),
                    "opt_init")

    def opt_step(self, theta_ptr, E_ptr, grad_ptr, stream=None):
        """One asynchronous optimiser step on device buffers (raw pointers)."""
        self._check(self._L.uccsd_opt_step(self._c, theta_ptr, E_ptr, grad_ptr,
                                           _stream_ptr(stream)), "opt_step")

    def gate(self, flag, target, timeout_s, stream):
        """Hold the work enqueued after this call on `stream` until the uint32
        at `flag` (a pinned CPU tensor, or a CUDA tensor) reaches `target`,
        at most `timeout_s` seconds (uccsd_gate_enqueue)."""
        self._check(self._L.uccsd_gate_enqueue(self._c, ctypes.c_void_p(flag.data_ptr()),
                                               int(target), int(timeout_s * 1e9),
                                               _stream_ptr(stream)), "gate_enqueue")

    def mark(self, stream):
        """Record the context's completion marker on `stream`
        (uccsd_stream_mark): mark_done() is True once the work enqueued
        there before it is done."""
        self._check(self._L.uccsd_stream_mark(self._c, _stream_ptr(stream)), "stream_mark")

    def mark_done(self):
        d = ctypes.c_int(0)
        self._check(self._L.uccsd_mark_done(self._c, ctypes.byref(d)), "mark_done")
        return bool(d.value)

    def zero_async(self, t, stream):
        """Zero the CUDA tensor t (contiguous) in order on `stream`
        (uccsd_zero_async)."""
        self._check(self._L.uccsd_zero_async(self._c, ctypes.c_void_p(t.data_ptr()),
                                             t.numel() * t.element_size(), _stream_ptr(stream)),
                    "zero_async")

    def gate_status(self, wait=True):
        """True once the gate was released, False while it waits; raises
        UCCSDError (code UCCSD_ERR_TIMEOUT = 5) if its time limit passed."""
        r = ctypes.c_int(0)
        self._check(self._L.uccsd_gate_status(self._c, 1 if wait else 0, ctypes.byref(r)),
                    "gate_status")
        return bool(r.value)

    def opt_history(self, cap=4096):
        E = np.zeros(max(cap, 1))
        n = ctypes.c_int(0)
        self._check(self._L.uccsd_opt_history(self._c, _f64p(E), cap, ctypes.byref(n)),
                    "opt_history")
        return E[:min(n.value, cap)].copy()

    def mp1_amplitudes(self, stream=None):
        """First-order amplitudes of the context's list (one device
        evaluation at theta = 0)."""
        t = np.zeros(max(self.K, 1))
        self._check(self._L.uccsd_mp1_amplitudes(self._c, _f64p(t), _stream_ptr(stream)),
                    "mp1_amplitudes")
        return t[:self.K].copy()

    def info(self):
        inf = Info()
        self._check(self._L.uccsd_info(self._c, ctypes.byref(inf)), "info")
        return inf.as_dict()


def energy_grad_batched(ctxs, thetas, E, grads=None, stream=None):
    """One evaluation per context in a single call (uccsd_energy_grad_batched):
    thetas a list of CUDA float64 tensors (K_i,), E a CUDA float64 tensor
    (len(ctxs),), grads a list of CUDA float64 tensors (K_i,) or None.  The
    contexts' evaluations overlap on the device; results are ordered on
    `stream`."""
    B = len(ctxs)
    if len(thetas) != B or E.numel() < B or (grads is not None and len(grads) != B):
        raise ValueError("one theta (and grad) per context, E of length len(ctxs)")
    for t in list(thetas) + ([E] + list(grads) if grads is not None else [E]):
        if not (t.is_cuda and t.dtype == torch_float64() and t.is_contiguous()):
            raise ValueError("thetas, E and grads must be contiguous CUDA float64 tensors")
    P = ctypes.c_void_p * max(B, 1)
    cs = P(*[c._c.value for c in ctxs])
    ts = P(*[t.data_ptr() for t in thetas])
    gs = P(*[g.data_ptr() for g in grads]) if grads is not None else None
    st = lib().uccsd_energy_grad_batched(cs, B, ts, E.data_ptr(), gs, _stream_ptr(stream))
    if st:
        msg = lib().uccsd_last_error(ctxs[0]._c).decode() if ctxs else ""
        raise UCCSDError(st, f"energy_grad_batched: {msg}")


def torch_float64():
    import torch
    return torch.float64


def make_context(n_orb, h, eri, e_core, n_alpha, n_beta, ijab=None, precision=FP64, device=0,
                 batch=1, trotter_order=1, n_slices=1, hbm_budget_bytes=0, layout=0):
    ctx = Context(device, precision, hbm_budget_bytes)
    ctx.set_hamiltonian(n_orb, h, eri, e_core)
    if layout:
        ctx.set_layout(layout)
    ctx.set_reference(n_alpha, n_beta)
    if ijab is None:
        ijab = build_uccsd_list(n_orb, n_alpha, n_beta)
    ctx.set_excitations(ijab, trotter_order, n_slices)
    if batch != 1:
        ctx.set_batch(batch)
    return ctx


from .autograd import UCCSDEnergy, uccsd_energy  # noqa: E402,F401
