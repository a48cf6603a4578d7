"""The stored expected values under tests/golden/ reproduce from the CPU
oracle (they are written by make_golden.py, which calls only the oracle),
and the 12-qubit reference energies satisfy what the mathematics fixes:
the theta = 0 energy is the closed-shell Hartree-Fock energy
2 sum_i h_ii + sum_ij [2 (ii|jj) - (ij|ji)] (Eq. 2 at the determinant of
Eq. 3), and the FCI energy lies below it."""
import json
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_8q_energy_and_gradient_reproduce():
    g = json.load(open(os.path.join(GOLDEN, "golden_8q.json")))
    w = synth.workload("8q")
    ex = oracle.excitations(4, 2, 2)
    th = synth.theta_uniform(len(ex), -0.1, 0.1, 1000)
    E, gr = oracle.energy_grad(4, w["h"], w["eri"], 0.0, 2, 2, ex, th)
    assert abs(E - g["E"]) < 1e-12
    assert np.max(np.abs(gr - np.array(g["grad"]))) < 1e-12


def test_golden_12q_reference_energies():
    g = json.load(open(os.path.join(GOLDEN, "golden_12q.json")))
    w = synth.workload("12q")
    h, eri = w["h"], w["eri"]
    occ = range(3)
    e_hf = 2 * sum(h[i, i] for i in occ) + sum(
        2 * eri[i, i, j, j] - eri[i, j, j, i] for i in occ for j in occ)
    assert abs(g["E_hf"] - e_hf) < 1e-11
    assert g["K"] == len(oracle.excitations(6, 3, 3))
    assert abs(g["E_fci"] - oracle.fci_energy(6, h, eri, 0.0, 3, 3)) < 1e-11
    assert g["E_fci"] < g["E_hf"]
