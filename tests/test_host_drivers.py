"""Host-side drivers on the CPU: L-BFGS bookkeeping and the FMO2 sum."""
import numpy as np

from paper_2402_17993_gb300.serving import fmo2_sum
from paper_2402_17993_gb300.vqe import LBFGS


def test_lbfgs_fixed_step_minimises_a_convex_quadratic():
    rng = np.random.default_rng(0)
    Q = rng.normal(size=(20, 20))
    A = Q @ Q.T / 20 + np.eye(20)
    b = rng.normal(size=20)
    x = np.zeros(20)
    opt = LBFGS(20, max_step=1.0, first_scale=0.1)
    for _ in range(60):
        g = A @ x - b
        x = opt.step(x, g)
    assert np.linalg.norm(A @ x - b) < 1e-6


def test_lbfgs_two_loop_equals_bfgs_inverse_on_stored_pairs():
    # with one stored pair, H g must satisfy the secant condition H y = s
    opt = LBFGS(3)
    s = np.array([0.3, -0.1, 0.2])
    y = np.array([0.5, 0.05, 0.4])
    opt.S, opt.Y = [s], [y]
    d = -opt.direction(y)
    assert np.allclose(d, s)


def test_lbfgs_skips_non_convex_pairs_and_caps_steps():
    opt = LBFGS(2, max_step=0.05)
    x = np.array([0.0, 0.0])
    x1 = opt.step(x, np.array([1.0, -1.0]))
    assert np.max(np.abs(x1 - x)) <= 0.05 + 1e-15
    opt.step(x1, np.array([2.0, -2.0]))  # y = (1, -1), s.y < 0: not stored
    assert len(opt.S) == 0


def test_fmo2_sum_matches_eq1_by_hand():
    # three fragments: E = (E12 + E13 + E23) - (3 - 2)(E1 + E2 + E3)
    mono = [-1.0, -2.0, -3.0]
    dim = [-3.5, -4.25, -5.0]
    assert fmo2_sum(mono, dim, 3) == (-3.5 - 4.25 - 5.0) - (-6.0)
