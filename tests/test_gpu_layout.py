"""The electron-sector state layout: the same arithmetic in the same order
as the full 2^n layout, so every energy and gradient is bitwise equal, and
equal to the oracle within the stated tolerances."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def uc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_17993_gb300 as uc
    uc.lib()
    return uc


def _pair(uc, w, ex, prec, **kw):
    args = (w["n_orb"], w["h"], w["eri"], 0.0, w["n_alpha"], w["n_beta"], ex)
    full = uc.make_context(*args, precision=prec, **kw)
    sect = uc.make_context(*args, precision=prec, layout=uc.LAYOUT_SECTOR, **kw)
    return full, sect


@pytest.mark.parametrize("name", ["8q", "12q", "18q"])
@pytest.mark.parametrize("prec", [0, 1])
def test_sector_layout_is_bitwise_equal_to_full_layout(uc, oracle_mod, name, prec):
    w = synth.workload(name)
    ex = oracle_mod.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
    B = 4
    th = np.stack([synth.theta_normal(len(ex), 0.05, 1002 + b) for b in range(B)])
    full, sect = _pair(uc, w, ex, prec, batch=B)
    assert sect.info()["layout"] == uc.LAYOUT_SECTOR
    assert sect.info()["device_bytes"] < full.info()["device_bytes"]
    Ef, gf = full.energy_grad_batch(th)
    Es, gs = sect.energy_grad_batch(th)
    assert np.array_equal(Ef, Es) and np.array_equal(gf, gs)
    # energy-only evaluation leaves the state: identical 2^n vectors
    full.energy(th[1])
    sect.energy(th[1])
    assert np.array_equal(full.state(), sect.state())
    if name != "18q":
        E0, g0 = oracle_mod.energy_grad(w["n_orb"], w["h"], w["eri"], 0.0, w["n_alpha"],
                                        w["n_beta"], ex, th[0])
        tol = 1e-10 if prec == 0 else 1e-5
        assert abs(Es[0] - E0) < tol and np.max(np.abs(gs[0] - g0)) < tol
    # the Trotter-free path and the first-order amplitudes run in both layouts
    assert full.energy_trotter_free(th[2]) == sect.energy_trotter_free(th[2])
    assert np.array_equal(full.mp1_amplitudes(), sect.mp1_amplitudes())
    full.close()
    sect.close()


def test_sector_layout_26q_golden(uc, oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "golden_26q.json")))
    w = synth.workload("26q")
    ex = oracle_mod.excitations(w["n_orb"], w["n_alpha"], w["n_beta"])
    th = synth.theta_normal(len(ex), 0.02, 1004)
    for prec, tol_e in ((0, 1e-10), (1, 1e-5)):
        ctx = uc.make_context(w["n_orb"], w["h"], w["eri"], 0.0, w["n_alpha"], w["n_beta"], ex,
                              precision=prec, layout=uc.LAYOUT_SECTOR)
        E, gr = ctx.energy_grad(th)
        assert abs(E - g["E"]) < tol_e
        gg = np.array(g["grad"])
        if prec == 0:
            assert np.max(np.abs(gr - gg)) < 1e-10
        else:
            assert np.max(np.abs(gr - gg) / np.maximum(1.0, np.abs(gg))) < 1e-5
        ctx.close()


def test_sector_layout_graph_replay_and_noalloc(uc, oracle_mod):
    import torch
    w = synth.workload("12q")
    ex = oracle_mod.excitations(6, 3, 3)
    th = synth.theta_normal(len(ex), 0.05, 1001)
    full, sect = _pair(uc, w, ex, 1, batch=2)
    s = torch.cuda.Stream()
    t = torch.tensor(np.stack([th, 0.5 * th]), dtype=torch.float64, device="cuda")
    out = {}
    for tag, ctx in (("full", full), ("sect", sect)):
        E = torch.zeros(2, dtype=torch.float64, device="cuda")
        G = torch.zeros(2, len(ex), dtype=torch.float64, device="cuda")
        ctx.capture(t, E, G, s)
        ctx.replay(s)
        s.synchronize()
        out[tag] = (E.cpu().numpy().copy(), G.cpu().numpy().copy())
    assert np.array_equal(out["full"][0], out["sect"][0])
    assert np.array_equal(out["full"][1], out["sect"][1])
    # the no-allocation energy reads a caller's 2^n state in either layout's context
    sect.energy(th)
    psi = sect.state()
    dev = torch.tensor(np.stack([psi.real, psi.imag], axis=1).astype(np.float32),
                       device="cuda").contiguous()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = sect._L.uccsd_expectation_noalloc(sect._c, dev.data_ptr(), E.data_ptr(),
                                           uc._stream_ptr(torch.cuda.current_stream()))
    assert st == 0
    torch.cuda.synchronize()
    assert abs(E.item() - sect.energy(th)) < 1e-5
    full.close()
    sect.close()


def test_set_layout_call_order(uc):
    w = synth.workload("8q")
    ctx = uc.Context(0, uc.FP64)
    ctx.set_hamiltonian(4, w["h"], w["eri"], 0.0).set_reference(2, 2)
    with pytest.raises(uc.UCCSDError):
        ctx.set_layout(uc.LAYOUT_SECTOR)
    ctx.set_hamiltonian(4, w["h"], w["eri"], 0.0)
    with pytest.raises(uc.UCCSDError):
        ctx.set_layout(7)
    ctx.set_layout(uc.LAYOUT_SECTOR).set_reference(2, 2)
    ctx.close()
