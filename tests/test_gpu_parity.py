"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Tolerances (FP error budget of the two precisions, stated in the design):
  FP64 state:                 |dE| <= 1e-10 Ha, max |dg| <= 1e-10
  FP32 state, FP64 reductions |dE| <= 1e-5 Ha,  max |dg| <= 1e-5
Cases span several shared-memory tiles and runs (18 qubits), the whole
register of sizes 2..26 qubits, empty/single/ragged excitation lists,
higher Trotter orders, open shells and batches.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {0: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def uc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_17993_gb300 as uc
    uc.lib()
    return uc


def ctx_for(uc, w, prec, ijab=None, **kw):
    return uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                           ijab=ijab, precision=prec, **kw)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["8q", "12q"])
def test_energy_grad_small(uc, oracle_mod, name, prec):
    w = synth.workload(name)
    ex = oracle_mod.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
    theta = synth.theta_normal(len(ex), 0.3, 99)
    E0, g0 = oracle_mod.energy_grad(w["n_orb"], w["h"], w["eri"], 0.0, w["n_alpha"], w["n_beta"],
                                    ex, theta)
    ctx = ctx_for(uc, w, prec)
    E, g = ctx.energy_grad(theta)
    assert abs(E - E0) <= TOL[prec]
    assert np.max(np.abs(g - g0)) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_state_vector_8q_and_12q(uc, oracle_mod, prec):
    for name in ("8q", "12q"):
        w = synth.workload(name)
        ex = oracle_mod.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
        theta = synth.theta_normal(len(ex), 0.4, 5)
        E0, _, psi0, _ = oracle_mod.energy_grad(w["n_orb"], w["h"], w["eri"], 0.0, w["n_alpha"],
                                                w["n_beta"], ex, theta, grad=False, want_state=True)
        ctx = ctx_for(uc, w, prec)
        E = ctx.energy(theta)
        psi = ctx.state(0)
        tol = 1e-13 if prec == 0 else 2e-6
        assert np.max(np.abs(psi - psi0)) <= tol
        assert abs(E - E0) <= TOL[prec]


def test_8q_sweep_matches_golden(uc):
    gold = json.load(open(os.path.join(HERE, "golden", "golden_8q.json")))
    w = synth.workload("8q")
    ctx = ctx_for(uc, w, 0)
    theta0 = synth.theta_uniform(ctx.K, -0.1, 0.1, 1000)
    E, g = ctx.energy_grad(theta0)
    assert abs(E - gold["E"]) <= 1e-10
    assert np.max(np.abs(g - np.array(gold["grad"]))) <= 1e-10
    k = gold["sweep_k"]
    es = []
    for s in range(16):
        th = theta0.copy()
        th[k] += -math.pi + 2 * math.pi * s / 16
        es.append(ctx.energy(th))
    assert np.max(np.abs(np.array(es) - np.array(gold["sweep_E"]))) <= 1e-10
    F = np.fft.rfft(np.array(es)) / 16
    assert np.max(np.abs(F[3:])) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_18q_batch_matches_golden(uc, prec):
    """Dimer-scale 18 qubits: several compact tiles and shared-memory passes."""
    gold = json.load(open(os.path.join(HERE, "golden", "golden_18q.json")))
    w = synth.workload("18q")
    ctx = ctx_for(uc, w, prec, batch=len(gold["evals"]))
    th = np.stack([synth.theta_normal(gold["K"], 0.05, r["theta_seed"]) for r in gold["evals"]])
    E, g = ctx.energy_grad_batch(th)
    for b, r in enumerate(gold["evals"]):
        assert abs(E[b] - r["E"]) <= TOL[prec], (b, E[b] - r["E"])
        assert np.max(np.abs(g[b] - np.array(r["grad"]))) <= TOL[prec]
    inf = ctx.info()
    assert inf["n_adj_runs"] > 1  # several shared-memory passes and tiles


def test_batch_equals_single_bitwise(uc):
    w = synth.workload("12q")
    ctx = ctx_for(uc, w, 1, batch=5)
    th = np.stack([synth.theta_normal(ctx.K, 0.1, 300 + b) for b in range(5)])
    E, g = ctx.energy_grad_batch(th)
    for b in (0, 3):
        e1, g1 = ctx.energy_grad(th[b])
        assert e1 == E[b] and np.array_equal(g1, g[b])
    E2, g2 = ctx.energy_grad_batch(th)
    assert np.array_equal(E, E2) and np.array_equal(g, g2)


def test_theta_zero_is_hf_and_empty_list(uc, oracle_mod):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    e_hf = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, np.zeros(len(ex)),
                                  grad=False)[0]
    for prec in (0, 1):
        ctx = ctx_for(uc, w, prec)
        assert abs(ctx.energy(np.zeros(ctx.K)) - e_hf) <= TOL[prec]
        empty = ctx_for(uc, w, prec, ijab=np.zeros((0, 4), dtype=np.int32))
        E, g = empty.energy_grad(np.zeros(0))
        assert abs(E - e_hf) <= TOL[prec] and g.size == 0


@pytest.mark.parametrize("order,M", [(1, 3), (2, 1), (2, 2)])
def test_trotter_variants(uc, oracle_mod, order, M):
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    theta = synth.theta_normal(len(ex), 0.3, 7)
    E0, g0 = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, theta, order=order, M=M)
    ctx = ctx_for(uc, w, 0, trotter_order=order, n_slices=M)
    E, g = ctx.energy_grad(theta)
    assert abs(E - E0) <= 1e-10 and np.max(np.abs(g - g0)) <= 1e-10


@pytest.mark.parametrize("n_orb,na,nb,seed", [(1, 1, 0, 3), (2, 1, 1, 4), (3, 2, 1, 5),
                                              (5, 3, 1, 6), (7, 2, 3, 8), (8, 4, 4, 9)])
def test_register_sizes_and_open_shells(uc, oracle_mod, n_orb, na, nb, seed):
    h, eri, _ = synth.make_integrals(n_orb, n_orb + 1, seed)
    ex = oracle_mod.excitations(n_orb, na, nb)
    theta = synth.theta_normal(len(ex), 0.4, seed + 50)
    E0, g0 = oracle_mod.energy_grad(n_orb, h, eri, 0.3, na, nb, ex, theta)
    for prec in (0, 1):
        ctx = uc.make_context(n_orb, h, eri, 0.3, na, nb, precision=prec)
        E, g = ctx.energy_grad(theta)
        assert abs(E - E0) <= TOL[prec]
        if len(ex):
            assert np.max(np.abs(g - g0)) <= TOL[prec]


def test_ragged_and_reordered_lists(uc, oracle_mod):
    """Arbitrary subsets, repeated excitations and non-lexicographic order."""
    w = synth.workload("18q")
    ex = oracle_mod.excitations(9, 5, 5)
    rng = np.random.default_rng(0)
    sub = ex[rng.permutation(len(ex))[:97]]
    sub = np.concatenate([sub, sub[:5]])
    theta = synth.theta_normal(len(sub), 0.2, 4)
    E0, g0 = oracle_mod.energy_grad(9, w["h"], w["eri"], 0.0, 5, 5, sub, theta, sector=True)
    ctx = ctx_for(uc, w, 0, ijab=sub)
    E, g = ctx.energy_grad(theta)
    assert abs(E - E0) <= 1e-10 and np.max(np.abs(g - g0)) <= 1e-10


def test_size_consistency_on_gpu(uc, oracle_mod):
    hA, eA, _ = synth.make_integrals(3, 4, 101)
    hB, eB, _ = synth.make_integrals(3, 4, 202)
    A, B = [0, 2, 3], [1, 4, 5]
    h = np.zeros((6, 6))
    eri = np.zeros((6,) * 4)
    h[np.ix_(A, A)] = hA
    h[np.ix_(B, B)] = hB
    eri[np.ix_(A, A, A, A)] = eA
    eri[np.ix_(B, B, B, B)] = eB
    exA = oracle_mod.excitations(3, 1, 1)

    def remap(row, orbs):
        return tuple(-1 if v < 0 else 2 * orbs[v // 2] + v % 2 for v in row)

    rows = np.array([remap(r, A) for r in exA] + [remap(r, B) for r in exA], dtype=np.int32)
    thA = synth.theta_normal(len(exA), 0.5, 5)
    thB = synth.theta_normal(len(exA), 0.5, 6)
    cA = uc.make_context(3, hA, eA, 0.0, 1, 1)
    cB = uc.make_context(3, hB, eB, 0.0, 1, 1)
    cD = uc.make_context(6, h, eri, 0.0, 2, 2, ijab=rows)
    ED = cD.energy(np.concatenate([thA, thB]))
    assert abs(ED - (cA.energy(thA) + cB.energy(thB))) <= 1e-11


def test_autograd_function(uc):
    import torch
    w = synth.workload("12q")
    ctx = ctx_for(uc, w, 0)
    theta = torch.tensor(synth.theta_normal(ctx.K, 0.1, 1), device="cuda", dtype=torch.float64,
                         requires_grad=True)
    E = uc.uccsd_energy(theta, ctx)
    E.backward()
    e_h, g_h = ctx.energy_grad(theta.detach().cpu().numpy())
    assert abs(E.item() - e_h) == 0.0
    assert torch.equal(theta.grad.cpu(), torch.tensor(g_h))


def test_errors_are_reported(uc):
    w = synth.workload("8q")
    ctx = uc.Context(0, 0)
    with pytest.raises(uc.UCCSDError) as e:
        ctx.set_reference(2, 2)
    assert e.value.code == 4
    ctx.set_hamiltonian(4, w["h"], w["eri"]).set_reference(2, 2)
    with pytest.raises(uc.UCCSDError) as e:
        ctx.set_excitations(np.array([[4, -1, 0, -1]], dtype=np.int32))  # virtual -> occupied
    assert e.value.code == 1
    with pytest.raises(uc.UCCSDError) as e:
        ctx.set_excitations(np.array([[0, -1, 5, -1]], dtype=np.int32))  # spin flip
    assert e.value.code == 1
    small = uc.Context(0, 0, hbm_budget_bytes=4096)
    with pytest.raises(uc.UCCSDError) as e:
        small.set_hamiltonian(9, *synth.make_integrals(9, 4, 0)[:2])
        small.set_reference(5, 5).set_excitations(uc.build_uccsd_list(9, 5, 5))
    assert e.value.code == 6


@pytest.mark.slow
@pytest.mark.parametrize("prec", [1, 0])
def test_26q_matches_golden(uc, prec):
    gold_path = os.path.join(HERE, "golden", "golden_26q.json")
    if not os.path.exists(gold_path):
        pytest.skip("26-qubit golden values not generated")
    gold = json.load(open(gold_path))
    w = synth.workload("26q")
    ctx = ctx_for(uc, w, prec)
    th = synth.theta_normal(gold["K"], 0.02, 1004)
    E, g = ctx.energy_grad(th)
    assert abs(E - gold["E"]) <= TOL[prec], E - gold["E"]
    g0 = np.array(gold["grad"])
    assert np.max(np.abs(g - g0)) <= TOL[prec], np.max(np.abs(g - g0))


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_over_contexts_equals_single_calls(uc, prec):
    # one uccsd_energy_grad_batched call over fragments of different sizes
    # (one of them twice) gives bitwise the energies and gradients of the
    # single calls; energies-only form as well
    import torch
    ws = [synth.workload(n) for n in ("8q", "12q", "18q")]
    ctxs = [ctx_for(uc, w, prec) for w in ws]
    order = [0, 1, 2, 1]
    thetas = [synth.theta_normal(ctxs[i].K, 0.05, 600 + j) for j, i in enumerate(order)]
    single = []
    for j, i in enumerate(order):
        single.append(ctxs[i].energy_grad(thetas[j]))
    th_d = [torch.tensor(t, device="cuda", dtype=torch.float64) for t in thetas]
    E = torch.zeros(len(order), device="cuda", dtype=torch.float64)
    G = [torch.zeros(ctxs[i].K, device="cuda", dtype=torch.float64) for i in order]
    s = torch.cuda.Stream()
    uc.energy_grad_batched([ctxs[i] for i in order], th_d, E, G, stream=s)
    s.synchronize()
    for j in range(len(order)):
        assert E[j].item() == single[j][0], j
        assert np.array_equal(G[j].cpu().numpy(), single[j][1]), j
    E2 = torch.zeros(len(order), device="cuda", dtype=torch.float64)
    uc.energy_grad_batched([ctxs[i] for i in order], th_d, E2, None, stream=s)
    s.synchronize()
    assert torch.equal(E, E2)
    with pytest.raises(ValueError):
        uc.energy_grad_batched(ctxs[:2], th_d[:1], E)
