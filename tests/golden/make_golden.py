"""Write the stored expected values under tests/golden/ from the CPU oracle.

Calls only ``oracle`` and ``synth`` (never the CUDA library).  Each file
records the workload, the theta recipe and the oracle's FP64 energy and
adjoint gradient of the first-order (M = 1) Trotterised UCCSD ansatz
(Eq. 5, energy of Section 2.3).

    python tests/golden/make_golden.py [8q] [12q] [18q] [26q]
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _dump(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=1)


def golden_8q():
    w = synth.workload("8q")
    ex = oracle.excitations(4, 2, 2)
    theta0 = synth.theta_uniform(len(ex), -0.1, 0.1, 1000)
    E0, g0 = oracle.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, theta0)
    k = int(np.nonzero(ex[:, 1] >= 0)[0][0])
    sweep = []
    for s in range(16):
        th = theta0.copy()
        th[k] += -math.pi + 2 * math.pi * s / 16
        sweep.append(oracle.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, th, grad=False)[0])
    _dump("golden_8q.json", dict(
        workload="8 qubits, 4 electrons, 4 spatial orbitals, integrals seed 0, 6 Cholesky vectors",
        theta="U(-0.1, 0.1), xoshiro256** seed 1000",
        sweep="theta0 + phi_s e_k, k = first double, phi_s = -pi + 2 pi s / 16",
        sweep_k=k, E=E0, grad=g0.tolist(), sweep_E=sweep))


def golden_12q():
    """Reference energies of the 12-qubit VQE workload: the Hartree-Fock
    determinant (theta = 0) and the exact sector ground state (FCI by
    dense diagonalisation), the lower bound of every UCCSD energy."""
    w = synth.workload("12q")
    ex = oracle.excitations(6, 3, 3)
    E_hf = oracle.energy_grad(6, w["h"], w["eri"], 0.0, 3, 3, ex, np.zeros(len(ex)), grad=False)[0]
    E_fci = oracle.fci_energy(6, w["h"], w["eri"], 0.0, 3, 3)
    _dump("golden_12q.json", dict(
        workload="12 qubits, 6 electrons, 6 spatial orbitals, integrals seed 1, 10 Cholesky vectors",
        K=len(ex), E_hf=E_hf, E_fci=E_fci))


def golden_18q(n_theta=4):
    w = synth.workload("18q")
    ex = oracle.excitations(9, 5, 5)
    rows = []
    for b in range(n_theta):
        th = synth.theta_normal(len(ex), 0.05, 1002 + b)
        t = time.time()
        E, g = oracle.energy_grad(9, w["h"], w["eri"], 0.0, 5, 5, ex, th, sector=True)
        rows.append(dict(theta_seed=1002 + b, E=E, grad=g.tolist(), oracle_s=time.time() - t))
    _dump("golden_18q.json", dict(
        workload="18 qubits, 10 electrons, 9 spatial orbitals, integrals seed 2, 16 Cholesky vectors",
        theta="N(0, 0.05), xoshiro256** seed 1002 + b", K=len(ex), evals=rows))


def golden_26q():
    w = synth.workload("26q")
    ex = oracle.excitations(13, 6, 6)
    th = synth.theta_normal(len(ex), 0.02, 1004)
    t = time.time()
    E, g = oracle.energy_grad(13, w["h"], w["eri"], 0.0, 6, 6, ex, th, sector=True)
    _dump("golden_26q.json", dict(
        workload="26 qubits, 12 electrons, 13 spatial orbitals, integrals seed 4, 20 Cholesky vectors",
        theta="N(0, 0.02), xoshiro256** seed 1004", K=len(ex), E=E, grad=g.tolist(),
        oracle_s=time.time() - t, oracle_threads=oracle.num_threads()))


if __name__ == "__main__":
    which = sys.argv[1:] or ["8q", "12q", "18q", "26q"]
    for name in which:
        t = time.time()
        {"8q": golden_8q, "12q": golden_12q, "18q": golden_18q, "26q": golden_26q}[name]()
        print(name, "done in", round(time.time() - t, 1), "s", flush=True)
