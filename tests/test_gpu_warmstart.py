"""Learned warm start on the GPU: the MLP kernels against torch FP32, and CTMRG from a prediction."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2512_14414_gb300.warmstart import WarmStart, converge, env_tensor_sizes, harvest, ising_states

pytestmark = pytest.mark.gpu


def test_mlp_forward_matches_torch_fp32():
    # 3 x (Linear 1024 + GELU) + Linear at the D=2, chi=8 sizes, random weights, batch 8
    w = W.config("heis_d2_chi8")
    n_out = sum(env_tensor_sizes(w.Lx, w.Ly, w.D, w.d, w.chi))
    net = WarmStart(w.d * w.D ** 4, n_out, seed=3)
    A = torch.tensor(np.stack(ising_states(w, range(8))), device="cuda")
    y = net.predict(A)
    ref = net.reference(A)
    torch.cuda.synchronize()
    assert y.shape == (8, n_out)
    assert float((y - ref).norm() / ref.norm()) <= 1e-5


def test_warm_started_ctmrg_reaches_the_cold_start_fixed_point():
    w = W.config("heis_d2_chi8")
    A, Y, its, _ = harvest(w, ising_states(w, range(48)))
    net = WarmStart(A[0].numel(), Y.shape[1])
    losses = net.fit(A, Y, epochs=150)
    assert losses[-1] < losses[0]
    from paper_2512_14414_gb300 import CTM
    ctm = CTM(w.Lx, w.Ly, w.d, w.D, w.chi, [(t.x, t.y, t.kind, t.coupling, t.h) for t in w.terms])
    env0 = torch.tensor(np.concatenate([a.ravel() for s in W.initial_environment(w) for a in s]), device="cuda")
    for A_np in ising_states(w, range(5000, 5003)):
        At = torch.tensor(A_np, device="cuda")
        n0, E0, ok0 = converge(ctm, At, env0)
        pred = net.predict(At[None]).to(torch.float64)[0].contiguous()
        n1, E1, ok1 = converge(ctm, At, pred)
        assert ok0 and ok1, (n0, n1)
        assert abs(E1 - E0) <= 1e-7, (E0, E1)
