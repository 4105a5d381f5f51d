"""L-BFGS outer loop of the variational calculation (Sec. SLF, step iii; Eq. OptPro).

The paper minimises E(X) with L-BFGS using the reverse-mode gradient of Eq. AD.  This module is
the host-side driver: the limited-memory BFGS two-loop recursion (Nocedal & Wright, *Numerical
Optimization*, 2nd ed., Alg. 7.4 and 7.5) with a line search satisfying the strong Wolfe
conditions (ibid., Alg. 3.5 and 3.6, cubic interpolation in the zoom phase).  The paper gives no
hyperparameters; history m = 10, c1 = 1e-4, c2 = 0.9, at most 20 steps are the defaults here.

Every energy and gradient comes from the caller's ``fun`` (for the PEPS: ``CTM.grad`` on the
GPU); the work done here is a few vector operations on the flattened site tensors, in FP64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Tuple

import numpy as np

Fun = Callable[[np.ndarray], Tuple[float, np.ndarray]]


@dataclass
class Result:
    x: np.ndarray
    f: float
    g: np.ndarray
    n_iter: int
    n_eval: int
    history: List[float] = field(default_factory=list)  # f after every accepted step (f0 first)
    converged: bool = False
    message: str = ""


def _cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic interpolating (a, fa, ga) and (b, fb, gb); None if it has none."""
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - ga * gb
    if disc < 0.0:
        return None
    d2 = np.sign(b - a) * np.sqrt(disc)
    den = gb - ga + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def line_search(fun: Fun, x, f0, g0, p, c1=1e-4, c2=0.9, a1=1.0, a_max=1e3, max_eval=20):
    """Step length along p satisfying the strong Wolfe conditions (Alg. 3.5 with zoom, Alg. 3.6).

    Returns (alpha, f, g, n_eval); alpha = 0 if no acceptable step was found.
    """
    d0 = float(g0 @ p)
    if d0 >= 0.0:
        return 0.0, f0, g0, 0
    n = 0

    def phi(a):
        nonlocal n
        n += 1
        f, g = fun(x + a * p)
        return f, g, float(g @ p)

    def zoom(lo, flo, dlo, glo, hi, fhi, dhi):
        # invariant: lo satisfies sufficient decrease with the lowest f seen; (hi - lo) * dlo < 0
        while n < max_eval:
            a = _cubic_min(lo, flo, dlo, hi, fhi, dhi)
            lo_b, hi_b = min(lo, hi), max(lo, hi)
            margin = 0.1 * (hi_b - lo_b)
            if a is None or not (lo_b + margin <= a <= hi_b - margin):
                a = 0.5 * (lo + hi)
            fa, ga, da = phi(a)
            if fa > f0 + c1 * a * d0 or fa >= flo:
                hi, fhi, dhi = a, fa, da
            else:
                if abs(da) <= -c2 * d0:
                    return a, fa, ga
                if da * (hi - lo) >= 0.0:
                    hi, fhi, dhi = lo, flo, dlo
                lo, flo, dlo, glo = a, fa, da, ga
        # out of evaluations: the best point with sufficient decrease, if any
        return (lo, flo, glo) if lo > 0.0 else None

    a_prev, f_prev, d_prev, g_prev = 0.0, f0, d0, g0
    a = a1
    for i in range(max_eval):
        fa, ga, da = phi(a)
        if fa > f0 + c1 * a * d0 or (i > 0 and fa >= f_prev):
            z = zoom(a_prev, f_prev, d_prev, g_prev, a, fa, da)
            return (z[0], z[1], z[2], n) if z else (0.0, f0, g0, n)
        if abs(da) <= -c2 * d0:
            return a, fa, ga, n
        if da >= 0.0:
            z = zoom(a, fa, da, ga, a_prev, f_prev, d_prev)
            return (z[0], z[1], z[2], n) if z else (0.0, f0, g0, n)
        a_prev, f_prev, d_prev, g_prev = a, fa, da, ga
        a = min(2.0 * a, a_max)
        if n >= max_eval:
            break
    return 0.0, f0, g0, n


def lbfgs(fun: Fun, x0: np.ndarray, m: int = 10, max_iter: int = 20, gtol: float = 1e-10,
          c1: float = 1e-4, c2: float = 0.9, callback=None) -> Result:
    """Minimise fun (returning value and gradient) from x0 by L-BFGS with history m."""
    x = np.array(x0, dtype=np.float64).ravel().copy()
    f, g = fun(x)
    g = np.asarray(g, dtype=np.float64).ravel()
    n_eval = 1
    S: List[np.ndarray] = []
    Y: List[np.ndarray] = []
    hist = [float(f)]
    res = Result(x, float(f), g, 0, n_eval, hist)
    for it in range(max_iter):
        if np.linalg.norm(g) <= gtol:
            res.converged, res.message = True, "gradient below gtol"
            break
        # two-loop recursion: p = -H g
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(S), reversed(Y)):
            rho = 1.0 / float(y @ s)
            a = rho * float(s @ q)
            q -= a * y
            alphas.append((rho, a))
        gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1]) if S else 1.0 / max(np.linalg.norm(g), 1e-300)
        r = gamma * q
        for (s, y), (rho, a) in zip(zip(S, Y), reversed(alphas)):
            b = rho * float(y @ r)
            r += (a - b) * s
        p = -r
        alpha, f_new, g_new, ne = line_search(fun, x, f, g, p, c1=c1, c2=c2)
        n_eval += ne
        if alpha == 0.0:
            res.message = "line search found no step satisfying the Wolfe conditions"
            break
        g_new = np.asarray(g_new, dtype=np.float64).ravel()
        s = alpha * p
        y = g_new - g
        if float(s @ y) > 1e-300:  # curvature condition holds under strong Wolfe; guard rounding
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x = x + s
        f, g = float(f_new), g_new
        hist.append(f)
        res = Result(x, f, g, it + 1, n_eval, hist)
        if callback is not None:
            callback(res)
    res.x, res.f, res.g, res.n_eval, res.history = x, float(f), g, n_eval, hist
    if not res.message:
        res.message = "converged" if res.converged else "max_iter reached"
    return res


def optimize_peps(ctm, A0: np.ndarray, env0, n_iter: int, max_steps: int = 20, m: int = 10, callback=None,
                  gradient: str = "unrolled", conv_tol: float = 1e-10, max_ctm: int = 400):
    """L-BFGS on the site tensors of a PEPS with the GPU energy and gradient.

    ``A0``: (Lx*Ly, d, D, D, D, D) FP64 host array; ``env0``: the initial environment (device FP64).
    ``gradient="unrolled"``: every evaluation runs ``n_iter`` iterations from ``env0`` and
    differentiates through all of them (``CTM.grad``), so E(X) is one fixed function.
    ``gradient="fixed_point"``: every evaluation starts from the environment the previous one
    converged (the first from ``env0``), iterates until the spectrum change of an iteration is at
    most ``conv_tol`` (at most ``max_ctm`` iterations) and takes the fixed-point gradient of the
    converged energy (``CTM.grad_fixed_point``); E(X) is then the converged energy, defined up to
    the convergence tolerance.
    """
    import torch

    shape = A0.shape
    dev = env0.device
    state = {"env": env0}

    def fun_unrolled(x):
        A = torch.from_numpy(x.reshape(shape)).to(dev)
        ctm.init(A, env0)
        e, dA = ctm.grad(n_iter)
        return float(e[0]), dA.detach().cpu().numpy().ravel()

    def fun_fixed_point(x):
        A = torch.from_numpy(x.reshape(shape)).to(dev)
        ctm.init(A, state["env"])
        done = 0
        while done < max_ctm:
            delta = ctm.step(5)
            done += 5
            if 0.0 <= delta <= conv_tol:
                break
        e, dA, _, _ = ctm.grad_fixed_point(tol=max(conv_tol, 1e-10))
        state["env"] = ctm.get_env().clone()
        return float(e[0]), dA.detach().cpu().numpy().ravel()

    fun = fun_fixed_point if gradient == "fixed_point" else fun_unrolled
    return lbfgs(fun, A0.ravel(), m=m, max_iter=max_steps, callback=callback)


def main():
    """Optimise a workload's PEPS with the GPU energy and gradient; one JSON line per step."""
    import argparse
    import json
    import time

    import torch

    import workloads as W
    from .api import CTM

    ap = argparse.ArgumentParser(description="L-BFGS on the nested single-layer CTMRG energy")
    ap.add_argument("--workload", default="ss_d6_chi64")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--history", type=int, default=10)
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--n-iter", type=int, default=None)
    ap.add_argument("--gradient", default="unrolled", choices=["unrolled", "fixed_point"])
    ap.add_argument("--conv-tol", type=float, default=None,
                    help="spectrum-change tolerance of the fixed-point evaluations (default 1e-10 in FP64, "
                         "1e-6 in the mixed modes)")
    args = ap.parse_args()
    w = W.config(args.workload)
    n_iter = args.n_iter or w.n_iter
    ctm = CTM(w.Lx, w.Ly, w.d, w.D, w.chi, [(t.x, t.y, t.kind, t.coupling, t.h) for t in w.terms],
              precision=args.precision)
    env0 = torch.tensor(np.concatenate([a.ravel() for s in W.initial_environment(w) for a in s]),
                        dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()

    def report(res):
        print(json.dumps({"step": res.n_iter, "energy": res.f, "grad_norm": float(np.linalg.norm(res.g)),
                          "evaluations": res.n_eval, "elapsed_s": time.perf_counter() - t0}), flush=True)

    conv_tol = args.conv_tol if args.conv_tol is not None else (1e-10 if args.precision == "fp64" else 1e-6)
    res = optimize_peps(ctm, np.stack(w.tensors), env0, n_iter, max_steps=args.steps, m=args.history,
                        callback=report, gradient=args.gradient, conv_tol=conv_tol)
    print(json.dumps({"workload": w.name, "precision": args.precision, "gradient": args.gradient,
                      "n_iter": n_iter, "steps": res.n_iter,
                      "energy_start": res.history[0], "energy_end": res.f, "evaluations": res.n_eval,
                      "message": res.message, "elapsed_s": time.perf_counter() - t0}), flush=True)


if __name__ == "__main__":
    main()
