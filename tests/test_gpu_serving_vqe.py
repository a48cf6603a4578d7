"""GPU tests of the VQE driver (12-qubit workload) and the fragment server."""
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


def test_vqe_12q_lbfgs_to_gradient_tolerance(uc, oracle_mod):
    from paper_2402_17993_gb300 import vqe
    w = synth.workload("12q")
    e_fci = oracle_mod.fci_energy(6, w["h"], w["eri"], 0.0, 3, 3)
    res = {}
    for prec in (uc.FP64, uc.FP32_STATE):
        ctx = uc.make_context(6, w["h"], w["eri"], 0.0, 3, 3, precision=prec)
        E, theta, n_eval, gnorm = vqe.minimize(ctx, gtol=1e-6 if prec == uc.FP64 else 1e-3)
        res[prec] = (E, theta)
        e_hf = ctx.energy(np.zeros(ctx.K))
        assert E < e_hf
        assert E >= e_fci - 1e-9
        if prec == uc.FP64:
            assert gnorm < 1e-6
            # the converged point: the oracle agrees on energy and gradient
            E0, g0 = oracle_mod.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3,
                                            oracle_mod.excitations(6, 3, 3), theta)
            assert abs(E0 - E) < 1e-10 and np.linalg.norm(g0) < 1e-6
    assert abs(res[uc.FP64][0] - res[uc.FP32_STATE][0]) < 1e-4


def _requests(n, seed=7):
    from paper_2402_17993_gb300.serving import Request
    return [Request(d["r"], d["t_unit"], d["n_orb"], d["n_alpha"], d["n_beta"], d["h"], d["eri"],
                    d["e_core"]) for d in synth.stream_fragments(n, seed)]


@pytest.mark.parametrize("prec", [1, 0])
def test_server_result_is_the_same_alone_and_in_the_mix(uc, prec):
    from paper_2402_17993_gb300.serving import FragmentServer
    reqs = _requests(12)
    srv = FragmentServer(precision=prec, steps=6, max_active=12)
    cold, _ = srv.run(reqs, rate=None, keep_theta=True)
    # warm: pooled contexts and cached pair lists, so the solves overlap
    mixed, stats = srv.run(reqs, rate=None, keep_theta=True)
    assert stats["requests"] == 12 and stats["evals"] == 72
    # the solves really ran side by side: some admission-to-done intervals overlap
    spans = sorted((m.t_admit, m.t_done) for m in mixed)
    assert any(b[0] < a[1] for a, b in zip(spans, spans[1:]))
    for c, m in zip(cold, mixed):
        assert c.energies == m.energies and np.array_equal(c.theta, m.theta)
    for q, m in zip(reqs, mixed):
        alone, _ = srv.run([q], rate=None, keep_theta=True)
        a = alone[0]
        assert a.r == m.r
        assert a.energies == m.energies          # bitwise: no cross-fragment coupling
        assert np.array_equal(a.theta, m.theta)
    srv.close()
    # energies decrease from the HF value over the fixed L-BFGS steps
    assert all(r.energies[-1] <= r.energies[0] + 1e-9 for r in mixed)


def test_server_first_step_energy_matches_oracle_hf(uc, oracle_mod):
    from paper_2402_17993_gb300.serving import FragmentServer
    reqs = _requests(6, seed=11)
    srv = FragmentServer(precision=uc.FP64, steps=1, max_active=6)
    res, _ = srv.run(reqs)
    for q, r in zip(reqs, res):
        ex = oracle_mod.excitations(q.n_orb, q.n_alpha, q.n_beta)
        e0 = oracle_mod.energy_grad(q.n_orb, q.h, q.eri, q.e_core, q.n_alpha, q.n_beta, ex,
                                    np.zeros(len(ex)), grad=False)[0]
        assert abs(r.energies[0] - e0) < 1e-10
    srv.close()


def test_server_admission_respects_hbm_budget(uc):
    from paper_2402_17993_gb300.serving import FragmentServer, footprint_bytes
    reqs = _requests(10)
    big = max(footprint_bytes(q.n_orb, q.n_alpha, q.n_beta, 1) for q in reqs)
    srv = FragmentServer(precision=1, steps=3, max_active=10, hbm_budget=2 * big)
    res, stats = srv.run(reqs)
    assert stats["requests"] == 10
    assert stats["peak_hbm_reserved_bytes"] <= 2 * big
    assert stats["peak_hbm_device_bytes"] <= stats["peak_hbm_reserved_bytes"]
    assert stats["mean_active"] < 10  # the budget, not the slot count, limited concurrency
    srv.close()


def test_server_open_loop_latencies(uc):
    from paper_2402_17993_gb300.serving import FragmentServer
    reqs = _requests(16)
    srv = FragmentServer(precision=1, steps=4, max_active=16)
    res, stats = srv.run(reqs, rate=200.0)
    assert stats["requests"] == 16
    assert 0 < stats["p50_latency_ms"] <= stats["p99_latency_ms"]
    assert all(r.t_done >= r.t_arrive for r in res)
    srv.close()


def test_device_lbfgs_follows_the_host_lbfgs(uc):
    # the device optimiser (uccsd_opt_step) and the host LBFGS class take the
    # same steps from the same evaluations (FP64, 12 qubits, 8 steps)
    import torch
    from paper_2402_17993_gb300.vqe import LBFGS
    w = synth.workload("12q")
    ctx = uc.make_context(6, w["h"], w["eri"], 0.0, 3, 3)
    K = ctx.K
    ctx.opt_init(memory=10, max_step=0.2, first_scale=0.1, max_steps=8)
    th = torch.zeros(K, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    G = torch.zeros(K, dtype=torch.float64, device="cuda")
    opt = LBFGS(K)
    theta = np.zeros(K)
    s = torch.cuda.current_stream()
    for _ in range(8):
        ctx.energy_grad_device(th.view(1, -1), E, G.view(1, -1), s)
        ctx.opt_step(th.data_ptr(), E.data_ptr(), G.data_ptr(), s)
        Eh, gh = ctx.energy_grad(theta)
        theta = opt.step(theta, gh)
    torch.cuda.synchronize()
    assert np.max(np.abs(th.cpu().numpy() - theta)) < 1e-9
    hist = ctx.opt_history()
    assert len(hist) == 8 and hist[0] == ctx.energy(np.zeros(K))
    assert hist[-1] < hist[0]
    ctx.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_setup_on_a_caller_stream_is_the_synchronous_setup(uc, prec):
    # One context refilled with fragments of different shapes and integrals,
    # its set-up transfers enqueued on a caller stream without host waits
    # (pinned staging, buffers that only grow), gives bitwise the energies and
    # gradients of fresh contexts set up synchronously.
    import torch
    s = torch.cuda.Stream()
    reuse = uc.Context(0, prec)
    rng = np.random.default_rng(5)
    frags = synth.stream_fragments(7, seed=11)
    for i, d in enumerate(frags):
        reuse.set_setup_stream(None if i == len(frags) - 1 else s)  # last one synchronous again
        reuse.set_hamiltonian(d["n_orb"], d["h"], d["eri"], d["e_core"])
        reuse.set_reference(d["n_alpha"], d["n_beta"])
        reuse.set_excitations(uc.build_uccsd_list(d["n_orb"], d["n_alpha"], d["n_beta"]))
        th = rng.uniform(-0.1, 0.1, reuse.K)
        Ea, ga = reuse.energy_grad(th, stream=s)
        fresh = uc.make_context(d["n_orb"], d["h"], d["eri"], d["e_core"], d["n_alpha"],
                                d["n_beta"], precision=prec)
        Eb, gb = fresh.energy_grad(th)
        fresh.close()
        assert Ea == Eb and np.array_equal(ga, gb), (i, d["n_orb"])
    assert len({d["n_orb"] for d in frags}) > 1
    reuse.close()


def test_captured_vqe_step_is_the_eager_step(uc):
    # one captured graph (evaluation + device L-BFGS step), replayed, takes
    # bitwise the steps of the eager evaluation and optimiser calls
    import torch
    w = synth.workload("12q")
    res = []
    for captured in (False, True):
        ctx = uc.make_context(6, w["h"], w["eri"], 0.0, 3, 3, precision=uc.FP32_STATE)
        K = ctx.K
        if captured:
            with pytest.raises(uc.UCCSDError):  # needs opt_init first
                z = torch.zeros(2 * K + 1, dtype=torch.float64, device="cuda")
                ctx.capture_vqe_step(z[:K], z[2 * K:], z[K:2 * K], torch.cuda.Stream())
        ctx.opt_init(memory=10, max_step=0.2, first_scale=0.1, max_steps=6)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            th = torch.zeros(K, dtype=torch.float64, device="cuda")
            E = torch.zeros(1, dtype=torch.float64, device="cuda")
            G = torch.zeros(K, dtype=torch.float64, device="cuda")
            if captured:
                ctx.capture_vqe_step(th, E, G, s)
                for _ in range(6):
                    ctx.replay(s)
            else:
                for _ in range(6):
                    ctx.energy_grad_device(th.view(1, -1), E, G.view(1, -1), s)
                    ctx.opt_step(th.data_ptr(), E.data_ptr(), G.data_ptr(), s)
        s.synchronize()
        res.append((th.cpu().numpy(), ctx.opt_history()))
        ctx.close()
    assert len(res[0][1]) == 6
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_contexts_prepared_on_many_threads_are_independent(uc):
    # distinct contexts on distinct host threads: set-up (Jordan-Wigner
    # compile, plans, shared pair lists), capture and evaluation run
    # concurrently and give bitwise the results of one thread doing the same
    import threading

    import torch
    reqs = _requests(16, seed=5)

    def solve(q, out, i):
        torch.cuda.set_device(0)
        ctx = uc.Context(0, 1)
        ctx.set_hamiltonian(q.n_orb, q.h, q.eri, q.e_core)
        ctx.set_reference(q.n_alpha, q.n_beta)
        ctx.set_excitations(uc.build_uccsd_list(q.n_orb, q.n_alpha, q.n_beta))
        th = synth.theta_normal(ctx.K, 0.05, 300 + i)
        out[i] = [ctx.energy_grad(th) for _ in range(3)]
        ctx.close()

    serial = {}
    for i, q in enumerate(reqs):
        solve(q, serial, i)
    conc = {}
    for _ in range(3):
        ths = [threading.Thread(target=solve, args=(q, conc, i)) for i, q in enumerate(reqs)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for i in range(len(reqs)):
            for (e1, g1), (e2, g2) in zip(serial[i], conc[i]):
                assert e1 == e2 and np.array_equal(g1, g2), i


def test_threaded_preparation_gives_the_serial_results(uc):
    from paper_2402_17993_gb300.serving import FragmentServer
    reqs = _requests(20, seed=13)
    res = {}
    for workers in (0, 8):
        srv = FragmentServer(precision=1, steps=5, max_active=16, prep_workers=workers)
        res[workers], stats = srv.run(reqs, keep_theta=True)
        assert stats["requests"] == 20 and stats["prep_workers"] == workers
        srv.close()
    for a, b in zip(res[0], res[8]):
        assert a.r == b.r and a.energies == b.energies and np.array_equal(a.theta, b.theta)


def test_gated_lookahead_gives_the_same_solves(uc):
    # open loop: the next requests are prepared before they arrive and wait
    # behind device gates released at their arrival; every solve is bitwise
    # the one prepared at arrival
    from paper_2402_17993_gb300.serving import FragmentServer
    reqs = _requests(12, seed=17)
    srv = FragmentServer(precision=1, steps=4, max_active=12)
    plain, _ = srv.run(reqs, rate=400.0, keep_theta=True)
    srv.lookahead = 6
    gated, stats = srv.run(reqs, rate=400.0, keep_theta=True)
    assert stats["lookahead"] == 6 and stats["requests"] == 12
    assert stats["gates_gave_up"] == 0
    for a, b in zip(plain, gated):
        assert a.r == b.r and a.energies == b.energies and np.array_equal(a.theta, b.theta)
        assert b.t_done >= b.t_arrive
    srv.close()
