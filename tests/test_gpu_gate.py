"""Bounded device wait of the serving loop (uccsd_gate_enqueue /
uccsd_gate_status).  The failure is made on the host: the flag is never
written, the gate gives up after its time limit, reports UCCSD_ERR_TIMEOUT,
and the device and the context stay usable."""
import time

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


def _ctx(uc):
    w = synth.workload("12q")
    return uc.make_context(w["n_orb"], w["h"], w["eri"], w["e_core"], w["n_alpha"], w["n_beta"],
                           precision=uc.FP64)


def test_gate_holds_the_work_until_the_host_releases_it(uc):
    import torch
    ctx = _ctx(uc)
    K = ctx.K
    th = torch.tensor(synth.theta_normal(K, 0.05, 21), device="cuda").view(1, -1)
    E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    G = torch.zeros(1, K, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32).pin_memory()
    s = torch.cuda.Stream()
    ctx.gate(flag, 1, 5.0, s)
    ctx.energy_grad_device(th, E, G, s)
    done = torch.cuda.Event()
    done.record(s)
    time.sleep(0.05)
    assert not done.query()              # held by the gate
    assert ctx.gate_status(wait=False) is False
    flag[0] = 1                          # the request "arrives"
    assert ctx.gate_status(wait=True) is True
    s.synchronize()
    E_ref, g_ref = ctx.energy_grad(th[0].cpu().numpy())
    assert E.item() == E_ref and np.array_equal(G[0].cpu().numpy(), g_ref)


def test_gate_gives_up_after_its_time_limit(uc):
    import torch
    ctx = _ctx(uc)
    flag = torch.zeros(1, dtype=torch.int32).pin_memory()  # never written
    s = torch.cuda.Stream()
    t0 = time.perf_counter()
    ctx.gate(flag, 1, 0.2, s)
    with pytest.raises(uc.UCCSDError) as e:
        ctx.gate_status(wait=True)
    waited = time.perf_counter() - t0
    assert e.value.code == 5             # UCCSD_ERR_TIMEOUT
    assert 0.15 <= waited < 5.0
    # the device and the context are free afterwards
    th = synth.theta_normal(ctx.K, 0.05, 22)
    E1, g1 = ctx.energy_grad(th)
    ctx2 = _ctx(uc)
    E2, g2 = ctx2.energy_grad(th)
    assert E1 == E2 and np.array_equal(g1, g2)
    # a new gate on the same context works again
    flag[0] = 7
    ctx.gate(flag, 7, 1.0, s)
    assert ctx.gate_status(wait=True) is True


def test_gate_argument_checks(uc):
    import torch
    ctx = _ctx(uc)
    flag = torch.zeros(1, dtype=torch.int32).pin_memory()
    s = torch.cuda.Stream()
    with pytest.raises(uc.UCCSDError) as e:
        ctx.gate(flag, 1, 0.0, s)
    assert e.value.code == 1
    with pytest.raises(uc.UCCSDError) as e:
        ctx.gate(flag, 1, 11.0, s)
    assert e.value.code == 1
    with pytest.raises(uc.UCCSDError) as e:
        ctx.gate_status()
    assert e.value.code == 4
    ctx.gate(flag, 1, 2.0, s)
    with pytest.raises(uc.UCCSDError) as e:   # one gate at a time
        ctx.gate(flag, 1, 2.0, s)
    assert e.value.code == 4
    flag[0] = 1
    assert ctx.gate_status(wait=True) is True
