"""Host-side variational drivers over the library's energy and adjoint gradient.

The paper optimises the UCCSD amplitudes with derivative-free COBYLA and
Powell (Section 2.3).  With the adjoint gradient available, these drivers use
limited-memory BFGS instead:

* ``LBFGS`` -- the two-loop recursion of Nocedal and Wright (Numerical
  Optimization, Algorithm 7.4) with a fixed step and no line search, so one
  optimiser step costs exactly one energy + gradient evaluation (the fragment
  serving loop runs a fixed number of such steps per solve).
* ``minimize`` -- scipy's L-BFGS-B on the same energy/gradient, to a gradient
  norm tolerance (the 12-qubit VQE workload).

All arithmetic here is host bookkeeping on K-vectors; every energy and
gradient comes from the CUDA library.
"""
from __future__ import annotations

import numpy as np


class LBFGS:
    """Fixed-step L-BFGS: theta <- theta + d with d = -H_k g (two-loop
    recursion, memory m, initial scaling s.y / y.y).  Pairs with
    s.y <= 0 are not stored.  The step is capped at `max_step` in the
    max-norm; the first step is -first_scale * g."""

    def __init__(self, K: int, m: int = 10, max_step: float = 0.2, first_scale: float = 0.1):
        self.K = K
        self.m = m
        self.max_step = max_step
        self.first_scale = first_scale
        self.S: list[np.ndarray] = []
        self.Y: list[np.ndarray] = []
        self.prev_theta = None
        self.prev_g = None

    def direction(self, g: np.ndarray) -> np.ndarray:
        if not self.S:
            return -self.first_scale * g
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(self.S), reversed(self.Y)):
            rho = 1.0 / float(y @ s)
            a = rho * float(s @ q)
            alphas.append((rho, a))
            q -= a * y
        s, y = self.S[-1], self.Y[-1]
        r = (float(s @ y) / float(y @ y)) * q
        for (s, y), (rho, a) in zip(zip(self.S, self.Y), reversed(alphas)):
            b = rho * float(y @ r)
            r += (a - b) * s
        return -r

    def step(self, theta: np.ndarray, g: np.ndarray) -> np.ndarray:
        if self.prev_theta is not None:
            s = theta - self.prev_theta
            y = g - self.prev_g
            if float(s @ y) > 1e-16 * max(1.0, float(y @ y)):
                self.S.append(s)
                self.Y.append(y)
                if len(self.S) > self.m:
                    self.S.pop(0)
                    self.Y.pop(0)
        d = self.direction(g)
        mx = float(np.max(np.abs(d))) if d.size else 0.0
        if mx > self.max_step:
            d *= self.max_step / mx
        self.prev_theta = theta.copy()
        self.prev_g = g.copy()
        return theta + d


def minimize(ctx, theta0=None, gtol: float = 1e-6, maxiter: int = 1000, trotter_free: bool = False):
    """VQE by scipy L-BFGS-B with the adjoint gradient until the gradient
    2-norm is below gtol.  trotter_free: optimise exp(sum theta G)|HF>
    (Eq. 3 without Trotterisation) instead of the context's Trotter product.
    Returns (E, theta, n_evals, grad_norm)."""
    import scipy.optimize

    K = ctx.K
    theta0 = np.zeros(K) if theta0 is None else np.asarray(theta0, dtype=np.float64)
    n_eval = [0]
    last = {}

    eg = ctx.energy_grad_trotter_free if trotter_free else ctx.energy_grad

    def fun(th):
        E, g = eg(th)
        n_eval[0] += 1
        last["g"] = g
        return E, g

    res = scipy.optimize.minimize(fun, theta0, jac=True, method="L-BFGS-B",
                                  options={"maxiter": maxiter, "gtol": gtol / np.sqrt(max(K, 1)),
                                           "ftol": 1e-15, "maxcor": 10})
    E, g = eg(res.x)
    return float(E), res.x, n_eval[0] + 1, float(np.linalg.norm(g))
