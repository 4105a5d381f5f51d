"""Fixed-point (implicit) gradient of the converged CTMRG energy (oracle, FP64).

Test infrastructure only: plain torch-CPU autograd, no blocking or fusion.

The Discussion section proposes computing the gradient from a given or
approximate fixed-point environment instead of differentiating through the
whole chain of CTMRG iterations (Eq. AD).  Write one CTMRG iteration
(left, right, up, down moves, Fig. CTMRG) as env' = f(A, env) and the energy
(Eq. ExpH) as e(A, env).  At a converged environment env* = f(A, env*) the
energy of the state is E(A) = e(A, env*(A)), and differentiating the fixed
point condition gives

    dE/dA = de/dA + lam df/dA,   lam = de/denv (I - df/denv)^{-1}
                                     = sum_k de/denv (df/denv)^k,

so lam is accumulated by repeated vector-Jacobian products through the one
recorded iteration at env*:  v_0 = de/denv,  dE/dA += v_k df/dA,
v_{k+1} = v_k df/denv, until the added term is below ``tol`` relative to the
running sum (the Neumann series converges when the spectral radius of
df/denv is below one, which is what makes env* an attracting fixed point).
In FP64 the terms fall geometrically (about tenfold per 10 products at
D=2, chi=8) down to a rounding floor near 1e-11 of the sum, so ``tol`` sits
above that floor.

This needs env* to be a fixed point element by element, not only up to a
gauge: the sign gauge of the projector SVD (``ctmrg._sign_gauge``) fixes the
one freedom the iteration has for non-degenerate spectra.

Parity: pinned by tests/test_oracle_pins.py (central finite differences of
the converged energy, with every perturbed state re-converged; the unrolled
gradient from env* over the same number of iterations; Euler's relation).
"""
from __future__ import annotations

import numpy as np
import torch

from .ctmrg import SLOTS, ctmrg, from_ring_arrays
from .energy import energy
from .nested import DT, nested_cell


def _flat(env):
    return [env[k][i][j] for k in SLOTS for i in range(len(env[k])) for j in range(len(env[k][0]))]


def fixed_point_energy_grad(As_np, Lx, Ly, chi, terms, env_star, max_adj=200, tol=1e-10):
    """E and dE/dA at the fixed point ``env_star`` (per-site ring arrays).

    Returns (E, [dE/dA_p as numpy arrays], n_adj, residual) where n_adj is the
    number of vector-Jacobian products taken and residual is
    ||f(A, env*) - env*|| / ||env*|| (how far env_star is from a fixed point).
    """
    As = [torch.tensor(np.asarray(a), dtype=DT, requires_grad=True) for a in As_np]
    grid = nested_cell(As, Lx, Ly)
    env = from_ring_arrays(env_star, len(grid), len(grid[0]))
    for k in SLOTS:
        for row in env[k]:
            for j in range(len(row)):
                row[j] = row[j].detach().clone().requires_grad_(True)
    leaves = _flat(env)
    E = energy(As, Lx, Ly, env, terms, grid=grid)
    g = torch.autograd.grad(E, As + leaves, allow_unused=True)
    dA = [torch.zeros_like(a) if x is None else x.clone() for a, x in zip(As, g[:len(As)])]
    v = [torch.zeros_like(t) if x is None else x for t, x in zip(leaves, g[len(As):])]
    out = _flat(ctmrg(grid, chi, 1, env=env))
    num = sum(float((o.detach() - l.detach()).pow(2).sum()) for o, l in zip(out, leaves))
    den = sum(float(l.detach().pow(2).sum()) for l in leaves)
    n_adj = 0
    for n_adj in range(1, max_adj + 1):
        h = torch.autograd.grad(out, As + leaves, grad_outputs=v, retain_graph=True, allow_unused=True)
        step = 0.0
        for p in range(len(As)):
            if h[p] is not None:
                dA[p] += h[p]
                step += float(h[p].pow(2).sum())
        v = [torch.zeros_like(t) if x is None else x for t, x in zip(leaves, h[len(As):])]
        total = sum(float(x.pow(2).sum()) for x in dA)
        if step <= tol * tol * total:
            break
    return float(E.detach()), [x.detach().numpy().copy() for x in dA], n_adj, (num / den) ** 0.5


def converge(As_np, Lx, Ly, chi, env0, tol=1e-13, max_iter=2000, chunk=10):
    """Iterate CTMRG from ``env0`` until one iteration changes the environment by at most ``tol``
    (relative, element-wise); returns (env, iterations, residual)."""
    from .api import warm_environment
    env, done = env0, 0
    while done < max_iter:
        env = warm_environment(As_np, Lx, Ly, chi, chunk, env)
        done += chunk
        nxt = warm_environment(As_np, Lx, Ly, chi, 1, env)
        a = np.concatenate([x.ravel() for s in env for x in s])
        b = np.concatenate([x.ravel() for s in nxt for x in s])
        res = float(np.linalg.norm(a - b) / np.linalg.norm(a))
        env, done = nxt, done + 1
        if res <= tol:
            return env, done, res
    return env, done, res
