"""Learned warm start: an MLP that predicts the CTMRG environment of a PEPS from its site tensors.

The paper starts every CTMRG contraction from a fixed environment (Sec. SLF, step ii) and has
no learned initialisation; this module is an addition.  A network maps the flattened site
tensors (FP32) through three hidden layers (Linear 1024 + GELU) and a linear output layer to the
whole nested environment in the ring layout of ``include/ctm.h``, each tensor normalised to
unit Frobenius norm.  CTMRG then iterates from the prediction to the same fixed point as from the
standard initial environment, in fewer iterations when the prediction is close.

* inference: ``ctm_mlp_forward`` (the library's GEMMs + a fused bias/GELU kernel);
* training data: (A, converged environment) pairs harvested by running the GPU CTMRG to a
  spectrum change below ``tol`` from the standard initial environment;
* training: Adam on the mean-squared error of the normalised environment, on the GPU through the
  library's own kernels (``ctm_mlp_backward`` for the gradient, ``ctm_adam_step`` for the update);
  a network kept on the CPU trains with plain torch instead.  Training is an offline step, not
  part of the energy/gradient path.

The environment is gauge dependent; the projector construction (sorted singular vectors with a
sign rule) fixes its basis well enough for a regression target, and where it does not the
prediction is still a valid starting point: the fixed point reached does not depend on it.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import time
from typing import List, Sequence, Tuple

import numpy as np
import torch

from . import _lib
from .api import CTM, _check, _stream

HIDDEN = 1024
N_HIDDEN = 3


def env_tensor_sizes(Lx: int, Ly: int, D: int, d: int, chi: int) -> List[int]:
    """Element counts of the environment tensors in ring-layout order (sites row-major, 8 slots)."""
    import workloads as W
    return [int(np.prod(s)) for site in W.env_shapes(Lx, Ly, D, d, chi) for s in site]


def normalise_env(env: torch.Tensor, sizes: Sequence[int]) -> torch.Tensor:
    """Each tensor of a flat environment (last axis) divided by its Frobenius norm."""
    parts = torch.split(env, list(sizes), dim=-1)
    return torch.cat([p / p.norm(dim=-1, keepdim=True).clamp_min(1e-300) for p in parts], dim=-1)


class WarmStart:
    """The network: weights as torch tensors; inference and (on the GPU) training through libctm."""

    def __init__(self, n_in: int, n_out: int, hidden: int = HIDDEN, n_hidden: int = N_HIDDEN, seed: int = 0,
                 device: str = "cuda"):
        g = torch.Generator(device="cpu").manual_seed(seed)
        dims = [n_in] + [hidden] * n_hidden + [n_out]
        self.dims = dims
        self.W, self.b = [], []
        for k in range(len(dims) - 1):
            bound = 1.0 / np.sqrt(dims[k])  # torch.nn.Linear's default initialisation range
            self.W.append((torch.rand(dims[k + 1], dims[k], generator=g) * 2 - 1).mul_(bound).to(device))
            self.b.append((torch.rand(dims[k + 1], generator=g) * 2 - 1).mul_(bound).to(device))
        self.mean = torch.zeros(n_in, device=device)
        self.scale = torch.ones(n_in, device=device)

    def _inputs(self, A: torch.Tensor) -> torch.Tensor:
        x = A.reshape(A.shape[0], -1).to(torch.float32)
        return ((x - self.mean) / self.scale).contiguous()

    def predict(self, A: torch.Tensor) -> torch.Tensor:
        """A: (batch, ...) site tensors on the GPU -> (batch, n_out) FP32 environment, via libctm."""
        lib = _lib.load()
        x = self._inputs(A)
        batch = x.shape[0]
        y = torch.empty(batch, self.dims[-1], dtype=torch.float32, device=x.device)
        work = torch.empty(2 * batch * max(self.dims[1:-1] or [1]), dtype=torch.float32, device=x.device)
        n = len(self.dims) - 1
        dims = (ctypes.c_int * (n + 1))(*self.dims)
        Wp = (ctypes.c_void_p * n)(*[w.data_ptr() for w in self.W])
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in self.b])
        _check(lib.ctm_mlp_forward(ctypes.c_void_p(x.data_ptr()), batch, n, dims, Wp, bp,
                                   ctypes.c_void_p(work.data_ptr()), ctypes.c_void_p(y.data_ptr()), _stream()),
               "ctm_mlp_forward")
        return y

    def reference(self, A: torch.Tensor) -> torch.Tensor:
        """The same network in plain torch FP32 (for training and for checking the kernels)."""
        h = self._inputs(A)
        for k, (w, b) in enumerate(zip(self.W, self.b)):
            h = torch.nn.functional.linear(h, w, b)
            if k < len(self.W) - 1:
                h = torch.nn.functional.gelu(h)
        return h

    def loss_and_grad(self, x: torch.Tensor, target: torch.Tensor):
        """Mean-squared error and its gradient with respect to every W_k and b_k, through
        ``ctm_mlp_backward``.  x: (batch, n_in) normalised FP32 inputs on the GPU."""
        lib = _lib.load()
        x = x.to(torch.float32).contiguous()
        target = target.to(torch.float32).contiguous()
        batch = x.shape[0]
        n = len(self.dims) - 1
        dims = (ctypes.c_int * (n + 1))(*self.dims)
        nwork = lib.ctm_mlp_work_floats(batch, n, dims)
        if nwork < 0:
            raise ValueError("bad network shape")
        work = torch.empty(int(nwork), dtype=torch.float32, device=x.device)
        dW = [torch.empty_like(w) for w in self.W]
        db = [torch.empty_like(b) for b in self.b]
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        vp = ctypes.c_void_p
        _check(lib.ctm_mlp_backward(vp(x.data_ptr()), vp(target.data_ptr()), batch, n, dims,
                                    (vp * n)(*[w.data_ptr() for w in self.W]), (vp * n)(*[b.data_ptr() for b in self.b]),
                                    (vp * n)(*[g.data_ptr() for g in dW]), (vp * n)(*[g.data_ptr() for g in db]),
                                    vp(work.data_ptr()), vp(loss.data_ptr()), _stream()), "ctm_mlp_backward")
        return loss, dW, db

    def fit(self, A: torch.Tensor, Y: torch.Tensor, epochs: int = 300, lr: float = 1e-3,
            batch_size: int = 64, seed: int = 0) -> List[float]:
        """Adam on the mean-squared error between prediction and normalised target environments
        (beta1 0.9, beta2 0.999, eps 1e-8): libctm's kernels when the network is on the GPU."""
        x = A.reshape(A.shape[0], -1).to(torch.float32)
        self.mean = x.mean(0)
        self.scale = x.std(0).clamp_min(1e-6) if x.shape[0] > 1 else torch.ones_like(self.mean)
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        n = A.shape[0]
        if self.W[0].is_cuda:
            lib = _lib.load()
            params = self.W + self.b
            moments = [(torch.zeros_like(p), torch.zeros_like(p)) for p in params]
            step = 0
            for _ in range(epochs):
                perm = torch.randperm(n, generator=g)
                tot = 0.0
                for i in range(0, n, batch_size):
                    idx = perm[i:i + batch_size].to(A.device)
                    loss, dW, db = self.loss_and_grad(self._inputs(A[idx]), Y[idx])
                    step += 1
                    for p, gr, (m, v) in zip(params, dW + db, moments):
                        _check(lib.ctm_adam_step(ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(gr.data_ptr()),
                                                 ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                                 p.numel(), lr, 0.9, 0.999, 1e-8, step, _stream()), "ctm_adam_step")
                    tot += float(loss[0]) * len(idx)
                losses.append(tot / n)
            return losses
        params = [t.requires_grad_(True) for t in self.W + self.b]
        opt = torch.optim.Adam(params, lr=lr)
        for _ in range(epochs):
            perm = torch.randperm(n, generator=g)
            tot = 0.0
            for i in range(0, n, batch_size):
                idx = perm[i:i + batch_size].to(A.device)
                loss = torch.mean((self.reference(A[idx]) - Y[idx]) ** 2)
                opt.zero_grad()
                loss.backward()
                opt.step()
                tot += float(loss.detach()) * len(idx)
            losses.append(tot / n)
        for t in params:
            t.requires_grad_(False)
        return losses


def converge(ctm: CTM, A: torch.Tensor, env0: torch.Tensor, tol: float = 1e-8, max_iter: int = 300
             ) -> Tuple[int, float, bool]:
    """CTMRG from env0 until the spectrum change of an iteration is below tol.

    Returns (iterations, energy per site, converged)."""
    ctm.init(A, env0)
    for it in range(1, max_iter + 1):
        delta = ctm.step(1)
        if it >= 2 and 0.0 <= delta < tol:
            return it, float(ctm.energy()[0]), True
    return max_iter, float(ctm.energy()[0]), False


def harvest(w, states: Sequence[np.ndarray], tol: float = 1e-8, max_iter: int = 300):
    """(A, normalised converged environment, iterations, energy) for each state, from the standard
    initial environment of the workload."""
    import workloads as W
    ctm = CTM(w.Lx, w.Ly, w.d, w.D, w.chi, [(t.x, t.y, t.kind, t.coupling, t.h) for t in w.terms],
              precision="fp64")
    env0 = torch.tensor(np.concatenate([a.ravel() for s in W.initial_environment(w) for a in s]),
                        dtype=torch.float64, device="cuda")
    sizes = env_tensor_sizes(w.Lx, w.Ly, w.D, w.d, w.chi)
    As, Ys, its, Es = [], [], [], []
    for A in states:
        At = torch.tensor(np.asarray(A), dtype=torch.float64, device="cuda").contiguous()
        n, E, ok = converge(ctm, At, env0, tol, max_iter)
        env = ctm.get_env()
        As.append(At)
        Ys.append(normalise_env(env.to(torch.float32), sizes))
        its.append(n)
        Es.append(E)
    return torch.stack(As), torch.stack(Ys), its, Es


def ising_states(w, seeds: Sequence[int], K_range=(0.30, 0.42)) -> List[np.ndarray]:
    """Site-tensor stacks of the Ising-wave-function family (workloads.ising_site) with K drawn
    per state from K_range and one noise seed per site."""
    import workloads as W
    out = []
    for s in seeds:
        K = float(np.random.default_rng(10_000 + s).uniform(*K_range))
        out.append(np.stack([W.ising_site(1000 * s + k, w.d, w.D, K=K) for k in range(w.Lx * w.Ly)]))
    return out


def main():
    ap = argparse.ArgumentParser(description="train the warm-start MLP and compare CTMRG iterations")
    ap.add_argument("--workload", default="heis_d2_chi8")
    ap.add_argument("--train", type=int, default=256)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--tol", type=float, default=1e-8)
    args = ap.parse_args()
    import workloads as W
    w = W.config(args.workload)
    t = time.perf_counter()
    A, Y, it_tr, _ = harvest(w, ising_states(w, range(args.train)), args.tol)
    t_h = time.perf_counter() - t
    net = WarmStart(A[0].numel(), Y.shape[1])
    t = time.perf_counter()
    losses = net.fit(A, Y, epochs=args.epochs)
    t_f = time.perf_counter() - t
    ctm = CTM(w.Lx, w.Ly, w.d, w.D, w.chi, [(tm.x, tm.y, tm.kind, tm.coupling, tm.h) for tm in w.terms],
              precision="fp64")
    env0 = torch.tensor(np.concatenate([a.ravel() for s in W.initial_environment(w) for a in s]),
                        dtype=torch.float64, device="cuda")
    cold, warm, dE, tc, tw = [], [], [], 0.0, 0.0
    for A_np in ising_states(w, range(100_000, 100_000 + args.test)):
        At = torch.tensor(A_np, dtype=torch.float64, device="cuda")
        t = time.perf_counter()
        n0, E0, _ = converge(ctm, At, env0, args.tol)
        tc += time.perf_counter() - t
        t = time.perf_counter()
        pred = net.predict(At[None]).to(torch.float64)[0].contiguous()
        n1, E1, _ = converge(ctm, At, pred, args.tol)
        tw += time.perf_counter() - t
        cold.append(n0)
        warm.append(n1)
        dE.append(abs(E1 - E0))
    print(json.dumps({"workload": w.name, "train_states": args.train, "test_states": args.test, "tol": args.tol,
                      "harvest_s": t_h, "fit_s": t_f, "final_loss": losses[-1],
                      "iterations_cold_mean": float(np.mean(cold)), "iterations_warm_mean": float(np.mean(warm)),
                      "wall_cold_s": tc, "wall_warm_s": tw, "max_abs_dE": float(np.max(dE))}))


if __name__ == "__main__":
    main()
