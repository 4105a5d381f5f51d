"""The L-BFGS outer loop (Sec. SLF, step iii) on CPU: textbook test functions and the oracle."""
import numpy as np
import pytest

import workloads as W
from paper_2512_14414_gb300.lbfgs import lbfgs, line_search


def rosenbrock(x):
    f = (1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2
    g = np.array([-2 * (1 - x[0]) - 400 * x[0] * (x[1] - x[0] ** 2), 200 * (x[1] - x[0] ** 2)])
    return f, g


def test_rosenbrock_reaches_the_minimum():
    res = lbfgs(rosenbrock, np.array([-1.2, 1.0]), max_iter=200, gtol=1e-9)
    assert np.allclose(res.x, [1.0, 1.0], atol=1e-6), res
    assert all(b <= a for a, b in zip(res.history, res.history[1:]))  # monotone decrease


def test_convex_quadratic_minimiser_is_the_linear_solve():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((20, 20))
    H = M @ M.T + 20 * np.eye(20)
    b = rng.standard_normal(20)
    fun = lambda x: (0.5 * x @ H @ x - b @ x, H @ x - b)
    res = lbfgs(fun, np.zeros(20), m=10, max_iter=200, gtol=1e-11)
    assert np.allclose(res.x, np.linalg.solve(H, b), atol=1e-9)


@pytest.mark.parametrize("x0,p", [(0.0, 1.0), (10.0, -1.0), (0.0, 100.0)])
def test_line_search_step_satisfies_the_strong_wolfe_conditions(x0, p):
    fun = lambda x: ((x[0] - 3.0) ** 4 + (x[0] - 3.0) ** 2, np.array([4 * (x[0] - 3.0) ** 3 + 2 * (x[0] - 3.0)]))
    x = np.array([x0])
    f0, g0 = fun(x)
    pv = np.array([p])
    a, fa, ga, _ = line_search(fun, x, f0, g0, pv, c1=1e-4, c2=0.9)
    assert a > 0
    assert fa <= f0 + 1e-4 * a * float(g0 @ pv)
    assert abs(float(ga @ pv)) <= 0.9 * abs(float(g0 @ pv))


def test_lowers_the_oracle_energy_of_a_small_peps():
    # the real objective: E(A) of the nested single-layer CTMRG (oracle, D=2, chi=4, 3 iterations)
    from oracle.api import evaluate
    w = W.custom(1, 1, 2, 4, 3, seeds=[0], terms=W.heisenberg_terms_rotated())
    env0 = W.initial_environment(w)
    shape = (1,) + w.tensors[0].shape

    def fun(x):
        E, g = evaluate([x.reshape(shape)[0]], w.Lx, w.Ly, w.chi, w.n_iter, w.terms, env0=env0, grad=True)
        return E, np.asarray(g[0]).ravel()

    res = lbfgs(fun, np.stack(w.tensors).ravel(), max_iter=3)
    assert res.n_iter >= 1
    assert res.history[-1] < res.history[0] - 1e-4
    assert all(b <= a + 1e-12 for a, b in zip(res.history, res.history[1:]))


class _FakeCTM:
    """Stands in for the GPU handle: an 'environment' that relaxes towards a function of A by a
    factor 10 per iteration, and a quadratic energy whose gradient grad_fixed_point returns."""

    def __init__(self, target):
        import torch
        self.torch, self.target = torch, target
        self.inits, self.steps = [], 0

    def init(self, A, env):
        self.A, self.env = A.clone(), env.clone()
        self.inits.append(env.clone())

    def step(self, n):
        goal = self.A.flatten()[: self.env.numel()] + 1.0
        delta = 0.0
        for _ in range(n):
            new = goal + 0.1 * (self.env - goal)
            delta = float((new - self.env).abs().max())
            self.env = new
            self.steps += 1
        return delta

    def get_env(self):
        return self.env.clone()

    def grad_fixed_point(self, tol=1e-10):
        d = self.A - self.target
        return self.torch.tensor([float((d * d).sum())]), 2 * d, 7, 0.0


def test_fixed_point_driver_warm_starts_and_converges_each_evaluation():
    # optimize_peps(gradient="fixed_point"): every evaluation starts from the environment the previous
    # one converged, iterates until the spectrum change is below conv_tol, then takes the fixed-point
    # gradient; L-BFGS drives the quadratic to its minimum
    import torch
    from paper_2512_14414_gb300.lbfgs import optimize_peps
    target = torch.arange(6, dtype=torch.float64).reshape(1, 6) / 7.0
    ctm = _FakeCTM(target)
    env0 = torch.zeros(3, dtype=torch.float64)
    res = optimize_peps(ctm, np.zeros((1, 6)), env0, n_iter=50, max_steps=20, gradient="fixed_point",
                        conv_tol=1e-9)
    assert np.allclose(res.x, target.numpy().ravel(), atol=1e-6)
    assert torch.equal(ctm.inits[0], env0)
    assert len(ctm.inits) == res.n_eval >= 2
    # each later evaluation starts where the previous one ended (not from env0)
    assert not torch.equal(ctm.inits[1], env0)
    # iterations come in chunks of 5 until the change is below 1e-9 (10x contraction: 10 iterations)
    assert ctm.steps % 5 == 0 and ctm.steps >= 10 * res.n_eval
