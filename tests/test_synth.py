"""Seeded synthetic inputs: determinism and the symmetries the recipe states."""
import numpy as np

import synth


def test_integrals_deterministic_and_symmetric():
    h1, e1, c1 = synth.make_integrals(5, 6, 3)
    h2, e2, c2 = synth.make_integrals(5, 6, 3)
    assert h1.tobytes() == h2.tobytes() and e1.tobytes() == e2.tobytes() and c1 == c2
    assert np.array_equal(h1, h1.T)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.array_equal(e1, e1.transpose(perm))
    assert np.allclose(np.diag(h1), np.linspace(-2, -0.5, 5))
    # (pq),(rs) supermatrix is positive semidefinite
    ev = np.linalg.eigvalsh(e1.reshape(25, 25))
    assert ev.min() > -1e-12


def test_different_seeds_differ():
    a = synth.make_integrals(4, 6, 0)[0]
    b = synth.make_integrals(4, 6, 1)[0]
    assert not np.array_equal(a, b)


def test_theta_streams():
    t = synth.theta_uniform(1000, -0.1, 0.1, 1000)
    assert t.min() >= -0.1 and t.max() < 0.1
    n = synth.theta_normal(20000, 0.05, 1002)
    assert abs(n.std() - 0.05) < 0.002 and abs(n.mean()) < 0.002


def test_stream_mix():
    reqs = synth.stream_requests(512)
    mono = sum(1 for r in reqs if r["n_orb"] <= 6)
    assert 0.5 < mono / 512 < 0.7
    assert all(r["n_elec"] in (4, 6, 8, 10) for r in reqs)
    ts = [r["t_unit"] for r in reqs]
    assert ts == sorted(ts)
