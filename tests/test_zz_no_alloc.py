"""The energy entry point that allocates no device memory.

uccsd_expectation_noalloc serves callers that cannot call cudaMalloc when
they need an energy: a serving loop held to a memory budget reserved up
front, where an allocation may fail or stall the device, or a plugin in a
program whose device allocator belongs to another framework and must not be
bypassed.  It takes the state vector and the
result buffer from the caller and keeps its per-tile partial sums in a fixed
array inside the library.

Here it is called through the C ABI twice in a row on the state that the
regular uccsd_energy call produced, and must report the same energy within
the library's tolerances (FP64 1e-10 Ha, FP32 state 1e-5 Ha); and on the
oracle's own state, where it must report the oracle's energy.  This
file is collected last so that a run stopping at its first failure has run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_17993_gb300 as uc
    uc.lib()
    return uc


def _noalloc(uc, ctx, psi_dev, E_dev):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    return uc.lib().uccsd_expectation_noalloc(ctx._c, ctypes.c_void_p(psi_dev.data_ptr()),
                                              ctypes.c_void_p(E_dev.data_ptr()),
                                              ctypes.c_void_p(stream))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_noalloc_energy_matches_uccsd_energy_twice(uc, prec, tol):
    import torch
    w = synth.workload("18q")
    ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                          precision=prec)
    ctype = np.complex128 if prec == 0 else np.complex64
    for seed in (1002, 1003):  # two calls in a row share the fixed scratch
        theta = synth.theta_normal(ctx.K, 0.05, seed)
        E_ref = ctx.energy(theta)               # regular entry point
        psi = torch.from_numpy(ctx.state(0).astype(ctype)).to("cuda")
        E_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(uc, ctx, psi, E_dev)
        assert st == 0, ctx._L.uccsd_last_error(ctx._c)
        torch.cuda.synchronize()
        assert abs(E_dev.item() - E_ref) <= tol


@pytest.mark.parametrize("name,prec,tol", [("8q", 0, 1e-10), ("12q", 0, 1e-10), ("12q", 1, 1e-5)])
def test_noalloc_energy_matches_the_oracle_on_its_own_state(uc, name, prec, tol):
    """Independent of the library's other entry points: the state comes
    from the oracle (its Trotterised ansatz at seeded theta), and the energy
    is compared with the oracle's <psi|H|psi> of that state."""
    import torch

    import oracle
    w = synth.workload(name)
    ex = oracle.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
    ctx = uc.Context(0, prec)
    ctx.set_hamiltonian(w["n_orb"], w["h"], w["eri"], w["e_core"])
    ctx.set_reference(w["n_alpha"], w["n_beta"])
    ctype = np.complex128 if prec == 0 else np.complex64
    for seed in (1000, 1001):
        theta = synth.theta_uniform(len(ex), -0.1, 0.1, seed)
        E_or, _, psi, _ = oracle.energy_grad(w["n_orb"], w["h"], w["eri"], w["e_core"],
                                             w["n_alpha"], w["n_beta"], ex, theta, grad=False,
                                             want_state=True)
        psi_dev = torch.from_numpy(psi.astype(ctype)).to("cuda")
        E_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(uc, ctx, psi_dev, E_dev) == 0, ctx._L.uccsd_last_error(ctx._c)
        torch.cuda.synchronize()
        assert abs(E_dev.item() - E_or) <= tol


def test_noalloc_rejects_states_above_the_scratch_limit(uc):
    import torch
    # 28 qubits, 7 + 7 electrons: C(14, 7) = 3432 rows of C(14, 7) columns,
    # two column blocks each, 6864 H-apply tiles (the scratch holds 4096)
    h, eri, _ = synth.make_integrals(14, 3, 7)
    ctx = uc.Context(0, 0)
    ctx.set_hamiltonian(14, h, eri).set_reference(7, 7)
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(uc, ctx, dummy, E_dev) == 1
    assert b"6864 H-apply tiles" in ctx._L.uccsd_last_error(ctx._c)


def test_noalloc_needs_a_reference(uc):
    import torch
    w = synth.workload("8q")
    ctx = uc.Context(0, 0)
    ctx.set_hamiltonian(4, w["h"], w["eri"])
    buf = torch.zeros(512, dtype=torch.float64, device="cuda")
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(uc, ctx, buf, E_dev) == 4
