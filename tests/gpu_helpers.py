"""Shared set-up of the GPU tests: seeded inputs in the layouts of include/ctm.h."""
import functools

import numpy as np
import torch

import workloads as W


def env_flat(env0, device="cuda"):
    return torch.tensor(np.concatenate([a.ravel() for s in env0 for a in s]), dtype=torch.float64, device=device)


def site_stack(tensors, device="cuda"):
    return torch.tensor(np.stack(tensors), dtype=torch.float64, device=device)


def make_ctm(w, precision="fp64"):
    from paper_2512_14414_gb300 import CTM
    return CTM(w.Lx, w.Ly, w.d, w.D, w.chi, [(t.x, t.y, t.kind, t.coupling, t.h) for t in w.terms],
               precision=precision)


def gpu_energy_grad(w, n_iter, precision="fp64", env0=None):
    env0 = W.initial_environment(w) if env0 is None else env0
    ctm = make_ctm(w, precision)
    ctm.init(site_stack(w.tensors), env_flat(env0))
    e, dA = ctm.grad(n_iter)
    torch.cuda.synchronize()
    return float(e[0]), dA.cpu().numpy().reshape(len(w.tensors), *w.tensors[0].shape), ctm


def oracle_energy_grad(w, n_iter, env0=None, grad=True):
    from oracle.api import evaluate
    env0 = W.initial_environment(w) if env0 is None else env0
    return evaluate(w.tensors, w.Lx, w.Ly, w.chi, n_iter, w.terms, env0=env0, grad=grad)


@functools.lru_cache(maxsize=4)
def _warm(name, n_warm):
    from oracle.api import warm_environment
    w = W.config(name)
    return warm_environment(w.tensors, w.Lx, w.Ly, w.chi, n_warm, W.initial_environment(w))


def oracle_warm_env(w, n_warm):
    """The environment the oracle reaches after ``n_warm`` iterations from the workload's seeded
    random environment: the pre-converged start of an evaluation inside an optimisation.  Both
    sides then evaluate from it, so the input comes from the oracle, never from the CUDA path."""
    return _warm(w.name, n_warm)


def rel_l2(a, b):
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
