"""Host-side pieces of the learned warm start (no GPU): layout of the target and the network."""
import numpy as np
import torch

import workloads as W
from paper_2512_14414_gb300.warmstart import WarmStart, env_tensor_sizes, ising_states, normalise_env


def test_environment_sizes_follow_the_ring_layout():
    w = W.config("heis_d2_chi8")
    env = W.initial_environment(w)
    assert env_tensor_sizes(w.Lx, w.Ly, w.D, w.d, w.chi) == [a.size for s in env for a in s]


def test_normalised_environment_has_unit_tensors():
    sizes = [4, 6, 3]
    x = torch.tensor(np.random.default_rng(0).standard_normal((5, 13)))
    y = normalise_env(x, sizes)
    for part in torch.split(y, sizes, dim=-1):
        assert torch.allclose(part.norm(dim=-1), torch.ones(5, dtype=y.dtype))


def test_network_shapes_and_training_lowers_the_loss():
    w = W.config("heis_d2_chi8")
    A = torch.tensor(np.stack(ising_states(w, range(8))))
    net = WarmStart(A[0].numel(), 40, hidden=64, device="cpu")
    Y = torch.randn(8, 40)
    assert net.reference(A).shape == (8, 40)
    losses = net.fit(A, Y, epochs=60, lr=3e-3, batch_size=4)
    assert losses[-1] < 0.5 * losses[0]
