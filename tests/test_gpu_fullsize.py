"""Full-size and degenerate cases on the GPU, checked through what holds at any size.

* E(A) is homogeneous of degree 0 in the site tensors (Eq. ExpH is a ratio and every CTMRG
  tensor is normalised), so E(2A) = E(A), dE/dA at 2A is half the one at A, and the Euler
  relation <dE/dA, A> = 0 holds -- checked at the bench configuration (D=6, chi=64,
  50 iterations, TF32x3) and at D=9, chi=81, 60 iterations.
* A D=1 product state has a rank-one environment (the degenerate end of the projector step,
  which takes the full factorisation); its energy and gradient have a closed form.
"""
import copy
import json
import os

import numpy as np
import pytest
import torch

import workloads as W
from gpu_helpers import gpu_energy_grad

pytestmark = pytest.mark.gpu


# The mixed-mode gradient after 60 unrolled iterations is only ~1e-2 accurate, so the D=9 case is
# checked in FP64 (its TF32x3 Euler residual, 8e-3, is recorded with the precision results).
@pytest.mark.parametrize("name,precision,euler_tol", [("ss_d6_chi64", "tf32x3", 1e-3), ("heis_d9_chi81", "fp64", 1e-8)])
def test_full_size_scale_invariance_and_euler_relation(name, precision, euler_tol):
    w = W.config(name)
    E1, g1, _ = gpu_energy_grad(w, w.n_iter, precision=precision)
    w2 = copy.copy(w)
    w2.tensors = [2.0 * a for a in w.tensors]
    E2, g2, _ = gpu_energy_grad(w2, w.n_iter, precision=precision)
    A = np.stack(w.tensors)
    assert abs(E1 - E2) <= 1e-9, (E1, E2)
    assert np.linalg.norm(2.0 * g2 - g1) <= 1e-6 * np.linalg.norm(g1)
    assert abs(float((g1 * A).sum())) <= euler_tol * np.linalg.norm(g1) * np.linalg.norm(A)


def test_d1_product_state_matches_its_closed_form_on_the_gpu():
    rng = np.random.default_rng(11)
    hs = rng.standard_normal((4, 4))
    hs = hs + hs.T
    v = np.array([0.8, -0.45])
    terms = [W.Term(0, 0, W.BOND_H, 0.7, hs), W.Term(0, 0, W.BOND_V, 1.3, hs)]
    w = W.custom(1, 1, 1, 2, 4, seeds=[0], terms=terms)
    w.tensors = [W.product_site(v)]
    E, g, _ = gpu_energy_grad(w, w.n_iter)
    vt = torch.tensor(v, requires_grad=True)
    vv = torch.kron(vt, vt)
    Ec = (0.7 + 1.3) * (vv @ torch.tensor(hs) @ vv) / (vt @ vt) ** 2
    Ec.backward()
    assert abs(E - float(Ec.detach())) < 1e-12
    assert np.abs(g.reshape(-1) - vt.grad.numpy()).max() < 1e-10


def test_rotated_neel_state_on_the_gpu():
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
    w = W.custom(1, 1, 1, 2, 3, seeds=[0], terms=W.heisenberg_terms_rotated())
    w.tensors = [W.neel_rotated_site()]
    E, _, _ = gpu_energy_grad(w, w.n_iter)
    assert abs(E - golden["neel_rotated_D1_energy_per_site"]["value"]) < 1e-12
