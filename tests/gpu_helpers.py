"""Shared set-up of the GPU tests: seeded inputs in the layouts of include/ctm.h."""
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


def rel_l2(a, b):
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
