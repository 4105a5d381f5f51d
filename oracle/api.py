"""One-call oracle evaluations: E and dE/dA for a workload (FP64, torch CPU)."""
from __future__ import annotations

import numpy as np
import torch

from .ctmrg import ctmrg, from_ring_arrays, to_ring_arrays
from .energy import energy
from .nested import DT, double_cell, nested_cell


def evaluate(As_np, Lx, Ly, chi, n_iter, terms, env0=None, grad=True, layer="nested",
             spectra_log=None, per_bond=None):
    """Energy per site after ``n_iter`` CTMRG iterations from the environment ``env0``.

    ``env0`` is a list of per-site ring-convention arrays (see
    ``ctmrg.from_ring_arrays``); None means the trivial boundary.

    Returns (E, [dE/dA_p as numpy arrays] or None).  The gradient is full
    reverse mode through every iteration (Eq. AD), no fixed-point shortcut.
    """
    As = [torch.tensor(np.asarray(a), dtype=DT, requires_grad=grad) for a in As_np]
    with torch.set_grad_enabled(grad):
        grid = nested_cell(As, Lx, Ly) if layer == "nested" else double_cell(As, Lx, Ly)
        R, C = len(grid), len(grid[0])
        env = None if env0 is None else from_ring_arrays(env0, R, C)
        env = ctmrg(grid, chi, n_iter, env=env, spectra_log=spectra_log)
        E = energy(As, Lx, Ly, env, terms, layer=layer, grid=grid, per_bond=per_bond)
        if not grad:
            return float(E.detach()), None
        E.backward()
    return float(E.detach()), [a.grad.numpy().copy() for a in As]


def warm_environment(As_np, Lx, Ly, chi, n_iter, env0):
    """The environment after ``n_iter`` CTMRG iterations (Fig. CTMRG) from ``env0``, returned
    in the per-site ring convention of ``env0``.  The evaluations of an optimisation start from
    such a pre-converged environment (the better initial value of the Discussion section)."""
    As = [torch.tensor(np.asarray(a), dtype=DT) for a in As_np]
    with torch.no_grad():
        grid = nested_cell(As, Lx, Ly)
        env = ctmrg(grid, chi, n_iter, env=from_ring_arrays(env0, len(grid), len(grid[0])))
    return [[np.ascontiguousarray(a) for a in site] for site in to_ring_arrays(env)]


def evaluate_workload(w, grad=True, n_iter=None, env0="default", **kw):
    """Nested evaluation of a workload from its seeded initial environment."""
    import workloads
    if isinstance(env0, str) and env0 == "default":
        env0 = workloads.initial_environment(w)
    return evaluate(w.tensors, w.Lx, w.Ly, w.chi, w.n_iter if n_iter is None else n_iter,
                    w.terms, env0=env0, grad=grad, **kw)
