"""Order parameters on the GPU (ctm_magnetization, Eq. Mag1; ctm_plaquette_order, Eq. Mag2) against
the oracle on the same seeded inputs and against the closed forms of product and dimer states."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import env_flat, make_ctm, site_stack

pytestmark = pytest.mark.gpu


def _oracle_env(w, n_iter):
    import torch
    from oracle.ctmrg import ctmrg, from_ring_arrays
    from oracle.nested import nested_cell
    As = [torch.tensor(a) for a in w.tensors]
    grid = nested_cell(As, w.Lx, w.Ly)
    env = ctmrg(grid, w.chi, n_iter, env=from_ring_arrays(W.initial_environment(w), 2 * w.Ly, 2 * w.Lx))
    return As, grid, env


def _gpu(w, n_iter):
    ctm = make_ctm(w)
    ctm.init(site_stack(w.tensors), env_flat(W.initial_environment(w)))
    ctm.step(n_iter)
    return ctm


def test_magnetization_matches_the_oracle_heisenberg_d2():
    from oracle.observables import magnetization
    w = W.config("heis_d2_chi8")
    As, grid, env = _oracle_env(w, w.n_iter)
    m_ref, M_ref = magnetization(As, 1, 1, env, grid)
    m, M = _gpu(w, w.n_iter).magnetization()
    assert np.abs(m.cpu().numpy() - m_ref).max() <= 1e-10
    assert abs(float(M[0]) - M_ref) <= 1e-10


def test_order_parameters_match_the_oracle_shastry_sutherland_cell():
    from oracle.observables import magnetization, plaquette_order
    from oracle.energy import energy
    w = W.custom(2, 2, 2, 6, 3, seeds=[2, 3, 4, 5], terms=W.shastry_sutherland_terms(), name="ss_small")
    As, grid, env = _oracle_env(w, w.n_iter)
    m_ref, M_ref = magnetization(As, 2, 2, env, grid)
    per = []
    energy(As, 2, 2, env, w.terms, grid=grid, per_bond=per)
    a, b = W.shastry_sutherland_empty_plaquettes()
    ctm = _gpu(w, w.n_iter)
    m, M = ctm.magnetization()
    assert np.abs(m.cpu().numpy() - m_ref).max() <= 1e-10
    assert abs(float(M[0]) - M_ref) <= 1e-10
    assert abs(float(ctm.plaquette_order(a, b)[0]) - plaquette_order(per, a, b)) <= 1e-10


def test_closed_forms_product_neel_dimer():
    v = np.array([0.8, -0.45])
    w = W.custom(1, 1, 1, 2, 3, seeds=[0], terms=W.heisenberg_terms_rotated())
    w.tensors = [W.product_site(v)]
    m, M = _gpu(w, 3).magnetization()
    n2 = v @ v
    ref = np.array([v[0] * v[1], 0.0, 0.5 * (v[0] ** 2 - v[1] ** 2)]) / n2
    assert np.abs(m.cpu().numpy()[0] - ref).max() < 1e-12
    w.tensors = [W.neel_rotated_site()]
    assert abs(float(_gpu(w, 3).magnetization()[1][0]) - 0.5) < 1e-12
    sites = W.dimer_singlet_sites()
    wd = W.Workload("dimer", 2, 2, 2, 2, 8, 4, sites, W.shastry_sutherland_terms())
    ctm = _gpu(wd, 4)
    m, M = ctm.magnetization()
    assert float(m.abs().max()) < 1e-12 and float(M[0]) < 1e-12
    a, b = W.shastry_sutherland_empty_plaquettes()
    assert float(ctm.plaquette_order(a, b)[0]) < 1e-12


def test_argument_checks():
    from paper_2512_14414_gb300 import CTMError
    w = W.config("heis_d2_chi8")
    ctm = _gpu(w, 1)
    with pytest.raises(CTMError):
        ctm.plaquette_order([0, 5], [1])     # term index out of range
