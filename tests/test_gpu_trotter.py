"""GPU parity of the Trotter-schedule helpers through the C ABI: first-order
amplitudes and the magnitude ordering of Section 2.3, and the Trotter-error
extrapolation of Section 3.2 over device energies at M = 1..5 slices."""
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


@pytest.mark.parametrize("name", ["8q", "12q", "18q"])
def test_mp1_amplitudes_match_oracle(uc, oracle_mod, name):
    w = synth.workload(name)
    n_orb, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    ex = oracle_mod.excitations(n_orb, na, nb)
    want, _ = oracle_mod.mp1_amplitudes(n_orb, w["h"], w["eri"], 0.0, na, nb, ex)
    for prec, tol in ((uc.FP64, 1e-10), (uc.FP32_STATE, 1e-5)):
        ctx = uc.make_context(n_orb, w["h"], w["eri"], 0.0, na, nb, ex, precision=prec)
        got = ctx.mp1_amplitudes()
        err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
        assert err.max() < tol, (prec, err.max())
        ctx.close()


def test_magnitude_ordered_circuit_matches_oracle_12q(uc, oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    ctx = uc.make_context(6, w["h"], w["eri"], 0.0, 3, 3, ex)
    t = ctx.mp1_amplitudes()
    rows, perm = uc.magnitude_order(ex, t)
    # the device-derived order is a valid magnitude order of the oracle's amplitudes
    t_or, _ = oracle_mod.mp1_amplitudes(6, w["h"], w["eri"], 0.0, 3, 3, ex)
    assert sorted(perm.tolist()) == list(range(len(ex)))
    mags = np.abs(t_or[perm])
    assert np.all(mags[:-1] >= mags[1:] - 1e-9 * np.maximum(1.0, mags[1:]))
    # energy and gradient of the reordered circuit
    th = synth.theta_normal(len(ex), 0.05, 1001)[perm]
    ctx.set_excitations(rows)
    E, g = ctx.energy_grad(th)
    E0, g0 = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, rows, th)
    assert abs(E - E0) < 1e-10 and np.max(np.abs(g - g0)) < 1e-10
    # the order matters: the lexicographic circuit at the same amplitudes differs
    E_lex = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, th[np.argsort(perm)],
                                   grad=False)[0]
    assert abs(E - E_lex) > 1e-8
    ctx.close()


@pytest.mark.parametrize("order,beta", [(1, 1.0), (2, 2.0)])
def test_trotter_extrapolation_of_device_energies(uc, oracle_mod, order, beta):
    w = synth.workload("8q")
    ex = oracle_mod.excitations(4, 2, 2)
    th = synth.theta_normal(len(ex), 0.05, 1000)
    Ms = [1, 2, 3, 4, 5]
    E_dev, E_or = [], []
    for M in Ms:
        ctx = uc.make_context(4, w["h"], w["eri"], 0.0, 2, 2, ex, trotter_order=order, n_slices=M)
        E_dev.append(ctx.energy(th))
        ctx.close()
        E_or.append(oracle_mod.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, th, order=order,
                                           M=M, grad=False)[0])
    assert np.max(np.abs(np.array(E_dev) - np.array(E_or))) < 1e-10
    a, b, c = uc.trotter_extrapolate(Ms, E_dev)
    a0, b0, c0 = oracle_mod.trotter_extrapolate(Ms, E_or)
    assert abs(b - b0) < 1e-5 * b0 and abs(a - a0) < 1e-5 * abs(a0) and abs(c - c0) < 1e-8
    E_free, _ = oracle_mod.trotter_free_energy(4, w["h"], w["eri"], 0.0, 2, 2, ex, th)
    assert abs(b - beta) < 0.1 * beta
    assert abs(c - E_free) < 0.1 * abs(E_dev[-1] - E_free)


# --- Trotter-free ansatz exp(sum theta G)|HF> on the device (Eq. 3) ---

@pytest.mark.parametrize("name,std", [("8q", 0.3), ("12q", 0.05), ("12q", 0.3), ("18q", 0.05)])
def test_trotter_free_energy_and_state_match_oracle(uc, oracle_mod, name, std):
    w = synth.workload(name)
    n_orb, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    ex = oracle_mod.excitations(n_orb, na, nb)
    th = synth.theta_normal(len(ex), std, 1001)
    E0, psi0 = oracle_mod.trotter_free_energy_sector(n_orb, w["h"], w["eri"], 0.0, na, nb, ex, th)
    for prec, tol in ((uc.FP64, 1e-10), (uc.FP32_STATE, 1e-5)):
        ctx = uc.make_context(n_orb, w["h"], w["eri"], 0.0, na, nb, ex, precision=prec)
        E = ctx.energy_trotter_free(th)
        assert abs(E - E0) < tol, (prec, E - E0)
        if prec == uc.FP64:
            assert np.max(np.abs(ctx.state() - psi0)) < 1e-12
        ctx.close()


def test_trotter_free_equals_trotter_for_commuting_generators(uc, oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    used, pick = set(), []
    for k, r in enumerate(ex):
        q = {int(v) for v in r if v >= 0}
        if not q & used:
            used |= q
            pick.append(k)
    sub = ex[pick]
    th = synth.theta_normal(len(sub), 0.4, 5)
    ctx = uc.make_context(6, w["h"], w["eri"], 0.0, 3, 3, sub)
    assert abs(ctx.energy_trotter_free(th) - ctx.energy(th)) < 1e-12
    # empty list and theta = 0 give the reference determinant's energy
    E_hf = ctx.energy(np.zeros(len(sub)))
    assert abs(ctx.energy_trotter_free(np.zeros(len(sub))) - E_hf) < 1e-12
    ctx.set_excitations(np.zeros((0, 4), np.int32))
    assert abs(ctx.energy_trotter_free(np.zeros(0)) - E_hf) < 1e-12
    ctx.close()


def test_trotter_free_device_theta_and_reuse(uc, oracle_mod):
    import torch
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    th = synth.theta_normal(len(ex), 0.05, 1001)
    ctx = uc.make_context(6, w["h"], w["eri"], 0.0, 3, 3, ex, batch=4)
    E_host = ctx.energy_trotter_free(th)
    t_dev = torch.tensor(th, dtype=torch.float64, device="cuda")
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    st = ctx._L.uccsd_energy_trotter_free(ctx._c, t_dev.data_ptr(), 1, E_dev.data_ptr(),
                                          uc._stream_ptr(s))
    assert st == 0
    s.synchronize()
    assert E_dev.item() == E_host
    # the Trotterised evaluation still works afterwards, batch included
    E, g = ctx.energy_grad_batch(np.stack([th] * 4))
    E1, g1 = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, th)
    assert np.max(np.abs(E - E1)) < 1e-10 and np.max(np.abs(g - g1)) < 1e-10
    ctx.close()


@pytest.mark.parametrize("name,std", [("8q", 0.3), ("12q", 0.05)])
def test_trotter_free_gradient_matches_oracle(uc, oracle_mod, name, std):
    w = synth.workload(name)
    n_orb, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    ex = oracle_mod.excitations(n_orb, na, nb)
    th = synth.theta_normal(len(ex), std, 1001)
    E0, g0 = oracle_mod.trotter_free_energy_grad_sector(n_orb, w["h"], w["eri"], 0.0, na, nb, ex, th)
    for prec, tol in ((uc.FP64, 1e-10), (uc.FP32_STATE, 1e-5)):
        ctx = uc.make_context(n_orb, w["h"], w["eri"], 0.0, na, nb, ex, precision=prec)
        E, g = ctx.energy_grad_trotter_free(th)
        assert abs(E - E0) < tol
        err = np.abs(g - g0) / np.maximum(1.0, np.abs(g0))
        assert err.max() < tol, (prec, err.max())
        ctx.close()


def test_trotter_free_gradient_18q_sampled_against_central_differences(uc, oracle_mod):
    w = synth.workload("18q")
    ex = oracle_mod.excitations(9, 5, 5)
    th = synth.theta_normal(len(ex), 0.05, 1001)
    ctx = uc.make_context(9, w["h"], w["eri"], 0.0, 5, 5, ex)
    E, g = ctx.energy_grad_trotter_free(th)
    hstep = 1e-4
    for k in (0, 39, 40, 300, len(ex) - 1):
        tp, tm = th.copy(), th.copy()
        tp[k] += hstep
        tm[k] -= hstep
        ep = oracle_mod.trotter_free_energy_sector(9, w["h"], w["eri"], 0.0, 5, 5, ex, tp)[0]
        em = oracle_mod.trotter_free_energy_sector(9, w["h"], w["eri"], 0.0, 5, 5, ex, tm)[0]
        assert abs((ep - em) / (2 * hstep) - g[k]) < 1e-6
    ctx.close()


def test_trotter_free_gradient_equals_trotter_gradient_for_commuting_generators(uc, oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    used, pick = set(), []
    for k, r in enumerate(ex):
        q = {int(v) for v in r if v >= 0}
        if not q & used:
            used |= q
            pick.append(k)
    sub = ex[pick]
    th = synth.theta_normal(len(sub), 0.4, 5)
    ctx = uc.make_context(6, w["h"], w["eri"], 0.0, 3, 3, sub)
    E, g = ctx.energy_grad_trotter_free(th)
    Et, gt = ctx.energy_grad(th)
    assert abs(E - Et) < 1e-12 and np.max(np.abs(g - gt)) < 1e-11
    ctx.set_excitations(np.zeros((0, 4), np.int32))
    E0, g0 = ctx.energy_grad_trotter_free(np.zeros(0))
    assert g0.shape == (0,) and abs(E0 - ctx.energy(np.zeros(0))) < 1e-12
    ctx.close()
