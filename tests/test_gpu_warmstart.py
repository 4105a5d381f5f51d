"""Learned warm start on the GPU: the MLP forward against torch FP32, its backward and the Adam step
against the FP64 oracle, training through the library's kernels, and CTMRG from a prediction."""
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


def test_mlp_backward_matches_the_oracle():
    # loss and gradient of every W_k and b_k through ctm_mlp_backward (FP32 kernels) against the
    # FP64 oracle's chain rule, at the network's real sizes for D=2, chi=8 (3 x 1024 hidden), batch 8
    from oracle import mlp
    w = W.config("heis_d2_chi8")
    n_out = sum(env_tensor_sizes(w.Lx, w.Ly, w.D, w.d, w.chi))
    net = WarmStart(w.d * w.D ** 4, n_out, seed=4)
    A = torch.tensor(np.stack(ising_states(w, range(8))), device="cuda")
    x = net._inputs(A)
    target = torch.randn(8, n_out, generator=torch.Generator().manual_seed(9)).to("cuda")
    loss, dW, db = net.loss_and_grad(x, target)
    torch.cuda.synchronize()
    L, dWr, dbr = mlp.loss_and_grad(x.cpu().numpy(), target.cpu().numpy(), [t.cpu().numpy() for t in net.W],
                                    [t.cpu().numpy() for t in net.b])
    assert abs(float(loss[0]) - L) <= 1e-5 * L
    for k in range(len(dW)):
        g, gr = dW[k].cpu().numpy(), dWr[k]
        assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr), k
        g, gr = db[k].cpu().numpy(), dbr[k]
        assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr), k


def test_adam_step_matches_the_oracle():
    import ctypes
    from oracle import mlp
    from paper_2512_14414_gb300 import _lib
    from paper_2512_14414_gb300.api import _check, _stream
    rng = np.random.default_rng(11)
    p, g, m = (rng.standard_normal(5000).astype(np.float32) for _ in range(3))
    v = rng.random(5000).astype(np.float32)
    dev = [torch.tensor(a, device="cuda") for a in (p, g, m, v)]
    lib = _lib.load()
    _check(lib.ctm_adam_step(*[ctypes.c_void_p(t.data_ptr()) for t in dev], 5000, 1e-3, 0.9, 0.999, 1e-8, 3,
                             _stream()), "ctm_adam_step")
    torch.cuda.synchronize()
    # the hyperparameters reach the kernel as FP32 values: the oracle takes the same rounded values
    f32 = lambda c: float(np.float32(c))
    pr, mr, vr = mlp.adam_step(p, g, m, v, f32(1e-3), f32(0.9), f32(0.999), f32(1e-8), 3)
    assert np.allclose(dev[0].cpu().numpy(), pr, rtol=1e-6, atol=1e-7)
    assert np.allclose(dev[2].cpu().numpy(), mr, rtol=1e-6, atol=1e-7)
    assert np.allclose(dev[3].cpu().numpy(), vr, rtol=1e-6, atol=1e-7)
