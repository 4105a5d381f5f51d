"""Fixed-point gradient (ctm_grad_fixed_point, Discussion section) on the GPU against the oracle's.

The oracle converges the environment itself (one iteration changes it by at most 1e-13, element by
element) and sums the Neumann series of its own vector-Jacobian products; the GPU starts from that
environment, runs a few iterations of its own and sums the same series through its kernels.  Both
are the derivative of the converged energy E(A) = e(A, env*(A)), which the oracle's pins tie to
central finite differences of re-converged energies.
"""
import functools

import numpy as np
import pytest

import workloads as W
from gpu_helpers import env_flat, make_ctm, rel_l2, site_stack

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=2)
def _oracle(name):
    from oracle.fixed_point import converge, fixed_point_energy_grad
    w = W.config(name)
    env, _, res = converge(w.tensors, w.Lx, w.Ly, w.chi, W.initial_environment(w), tol=1e-13)
    assert res <= 1e-13
    E, g, _, _ = fixed_point_energy_grad(w.tensors, w.Lx, w.Ly, w.chi, w.terms, env)
    return env, E, g


@pytest.mark.parametrize("name", ["heis_d2_chi8", "heis_d4_chi32"])
def test_fixed_point_gradient_matches_the_oracle(name):
    w = W.config(name)
    env, Er, gr = _oracle(name)
    ctm = make_ctm(w, "fp64")
    ctm.init(site_stack(w.tensors), env_flat(env))
    ctm.step(5)
    e, dA, terms, res = ctm.grad_fixed_point()
    assert res <= 1e-9, res  # measured 2e-11 to 3e-11: the GPU's own fixed point, in its rounding
    assert terms < 200, terms
    assert abs(float(e[0]) - Er) <= 1e-10, (float(e[0]), Er)
    assert rel_l2(dA.cpu().numpy(), gr) <= 1e-5, rel_l2(dA.cpu().numpy(), gr)


def test_unrolled_gradient_from_the_fixed_point_approaches_it():
    # from env*, the unrolled reverse mode over n iterations is the series cut after n terms
    w = W.config("heis_d2_chi8")
    env, _, _ = _oracle("heis_d2_chi8")
    ctm = make_ctm(w, "fp64")
    A = site_stack(w.tensors)
    ctm.init(A, env_flat(env))
    ctm.step(5)
    e, dA, _, _ = ctm.grad_fixed_point()
    g = dA.cpu().numpy()
    ctm.init(A, ctm.get_env())
    eu, dAu = ctm.grad(60)
    assert abs(float(eu[0]) - float(e[0])) <= 1e-13
    assert rel_l2(dAu.cpu().numpy(), g) <= 1e-7
    # Euler's relation: E is invariant under A -> c A
    assert abs(float(np.sum(g * A.cpu().numpy()))) <= 1e-10 * np.linalg.norm(g) * np.linalg.norm(A.cpu().numpy())


def test_mixed_mode_fixed_point_gradient_matches_the_oracle():
    # TF32x3 contractions: the environment converges only to FP32 rounding, which bounds what the
    # series can resolve; the mixed-mode bars apply
    w = W.config("heis_d4_chi32")
    env, Er, gr = _oracle("heis_d4_chi32")
    ctm = make_ctm(w, "tf32x3")
    ctm.init(site_stack(w.tensors), env_flat(env))
    ctm.step(5)
    e, dA, terms, res = ctm.grad_fixed_point(tol=1e-6)
    assert res <= 1e-4, res
    assert abs(float(e[0]) - Er) <= 1e-6, (float(e[0]), Er)
    assert rel_l2(dA.cpu().numpy(), gr) <= 1e-3, rel_l2(dA.cpu().numpy(), gr)


def test_argument_checks():
    from paper_2512_14414_gb300.api import CTMError
    w = W.config("heis_d2_chi8")
    ctm = make_ctm(w, "fp64")
    with pytest.raises(CTMError):
        ctm.grad_fixed_point()  # before ctm_init
    ctm.init(site_stack(w.tensors), env_flat(W.initial_environment(w)))
    with pytest.raises(CTMError):
        ctm.grad_fixed_point(max_terms=0)
