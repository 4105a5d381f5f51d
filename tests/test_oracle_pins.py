"""The oracle pinned against things other than itself (CPU only).

* exact finite clusters (state vector vs nested vs double-layer networks),
* the variational bound from a Lanczos ground state,
* closed forms: D=1 product states, the Shastry-Sutherland dimer state,
* decoupled chains, whose energy follows from the MPS transfer matrix,
* single- vs double-layer CTMRG agreement (Appendix),
* the projector adjoint vs torch autograd of plain QR+SVD, and the full
  gradient vs central finite differences,
* invariants: scale, Euler relation, lattice rotation.
"""
import json
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import exact
from oracle.api import evaluate
from oracle.ctmrg import ctmrg, init_env, projectors, projectors_plain, from_ring_arrays, to_ring_arrays
from oracle.energy import energy
from oracle.nested import DT, nested_cell

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _env0(Lx, Ly, D, chi, d=2, seed=12345):
    w = W.Workload("t", Lx, Ly, d, D, chi, 0, [], [])
    return W.initial_environment(w, seed)


# ----------------------------------------------------------------------------- exact clusters
def test_finite_cluster_nested_and_double_equal_state_vector():
    rng = np.random.default_rng(3)
    D, d, Lx, Ly = 2, 2, 3, 2
    sites = [[torch.tensor(rng.standard_normal((d, D, D, D, D))) for _ in range(Lx)] for _ in range(Ly)]
    psi = exact.state_vector(sites)
    h = W.heisenberg_bond()
    for s1, s2 in exact.cluster_bonds(Lx, Ly):
        i, j = s1[1] * Lx + s1[0], s2[1] * Lx + s2[0]
        esv = exact.bond_expectation_sv(psi, h, i, j)
        for rdm in (exact.nested_bond_rdm, exact.double_bond_rdm):
            r = rdm(sites, s1, s2, d)
            e = float(torch.einsum("ab,ba", r, torch.tensor(h)) / torch.trace(r))
            assert abs(e - esv) < 1e-12


def test_state_vector_amplitude_by_brute_force():
    # 2x2 open cluster: amplitude = sum over all virtual indices of the product (Eq. PEPS)
    rng = np.random.default_rng(4)
    D, d = 2, 2
    T = [torch.tensor(rng.standard_normal((d, D, D, D, D))) for _ in range(4)]
    psi = exact.state_vector([[T[0], T[1]], [T[2], T[3]]])
    for s in np.ndindex(2, 2, 2, 2):
        amp = 0.0
        for a, b, c, e in np.ndindex(D, D, D, D):  # a: (0,0)-(1,0), b: (0,1)-(1,1), c: (0,0)-(0,1), e: (1,0)-(1,1)
            amp += float(T[0][s[0], 0, 0, a, c] * T[1][s[1], a, 0, 0, e] * T[2][s[2], 0, c, b, 0] * T[3][s[3], b, e, 0, 0])
        assert abs(amp - float(psi[s])) < 1e-12


def test_lanczos_matches_dense_and_bounds_peps_energy():
    h = W.heisenberg_bond()
    # dense diagonalisation of a 2x3 open cluster
    Lx, Ly = 3, 2
    n = Lx * Ly
    H = np.zeros((2**n, 2**n))
    for (x1, y1), (x2, y2) in exact.cluster_bonds(Lx, Ly):
        i, j = y1 * Lx + x1, y2 * Lx + x2
        for b in range(2**n):
            bits = [(b >> (n - 1 - k)) & 1 for k in range(n)]
            row = bits[i] * 2 + bits[j]
            for col in range(4):
                v = h[col, row]
                if v != 0.0:
                    nb = list(bits)
                    nb[i], nb[j] = col // 2, col % 2
                    H[int("".join(map(str, nb)), 2), b] += v
    e_dense = np.linalg.eigvalsh(H)[0]
    assert abs(exact.lanczos_ground(Lx, Ly, h) - e_dense) < 1e-9
    # variational bound on the 4x4 cluster for a random D=2 PEPS (rotated frame, same spectrum)
    rng = np.random.default_rng(5)
    A = torch.tensor(np.abs(rng.standard_normal((2, 2, 2, 2, 2))))
    sites = [[A] * 4 for _ in range(4)]
    psi = exact.state_vector(sites)
    hr = W.heisenberg_bond_rotated()
    esv = sum(exact.bond_expectation_sv(psi, hr, y1 * 4 + x1, y2 * 4 + x2)
              for (x1, y1), (x2, y2) in exact.cluster_bonds(4, 4))
    e0 = exact.lanczos_ground(4, 4, hr)
    assert esv >= e0 - 1e-9
    assert abs(exact.lanczos_ground(4, 4, h) - e0) < 1e-8   # rotation is unitary on a bipartite cluster


# ----------------------------------------------------------------------------- closed forms
def test_neel_rotated_product_state():
    A = W.neel_rotated_site()
    E, g = evaluate([A], 1, 1, 2, 3, W.heisenberg_terms_rotated(), env0=_env0(1, 1, 1, 2))
    assert abs(E - GOLDEN["neel_rotated_D1_energy_per_site"]["value"]) < 1e-12


def test_d1_product_state_energy_and_gradient_closed_form():
    rng = np.random.default_rng(11)
    hs = rng.standard_normal((4, 4))
    hs = hs + hs.T
    v = np.array([0.8, -0.45])
    terms = [W.Term(0, 0, W.BOND_H, 0.7, hs), W.Term(0, 0, W.BOND_V, 1.3, hs)]
    E, g = evaluate([W.product_site(v)], 1, 1, 2, 4, terms, env0=_env0(1, 1, 1, 2))
    vt = torch.tensor(v, requires_grad=True)
    vv = torch.kron(vt, vt)
    Ec = (0.7 + 1.3) * (vv @ torch.tensor(hs) @ vv) / (vt @ vt) ** 2
    Ec.backward()
    assert abs(E - float(Ec.detach())) < 1e-12
    assert np.abs(g[0].reshape(-1) - vt.grad.numpy()).max() < 1e-10


def test_dimer_singlet_state_exact():
    sites = W.dimer_singlet_sites()
    pb = []
    E, _ = evaluate(sites, 2, 2, 8, 6, W.shastry_sutherland_terms(), env0=_env0(2, 2, 2, 8),
                    grad=False, per_bond=pb)
    assert abs(E - GOLDEN["ss_dimer_singlet_energy_per_site"]["value"]) < 1e-12
    assert all(abs(e) < 1e-12 for e in pb[:8])
    assert all(abs(e - GOLDEN["ss_dimer_singlet_bond"]["value"]) < 1e-12 for e in pb[8:])


def test_dimer_peps_is_the_singlet_product_by_state_vector():
    # the D=2 construction on a 4x2 open strip: every J' pair (A-F, B-C') inside it is a singlet
    A, B, C, F = [torch.tensor(t) for t in W.dimer_singlet_sites()]
    sites = [[A, B, A, B], [C, F, C, F]]
    psi = exact.state_vector(sites)
    h = W.heisenberg_bond()
    # A(0,0)-F(1,1) and A(2,0)-F(3,1) are complete singlets inside the strip
    for (x1, y1, x2, y2) in ((0, 0, 1, 1), (2, 0, 3, 1)):
        assert abs(exact.bond_expectation_sv(psi, h, y1 * 4 + x1, y2 * 4 + x2) + 0.75) < 1e-12


def test_decoupled_chains_match_transfer_matrix():
    rng = np.random.default_rng(5)
    D = 2
    A = np.zeros((2, D, D, D, D))
    A[:, :, 0, :, 0] = np.abs(rng.standard_normal((2, D, D)))
    M = A[:, :, 0, :, 0]
    T = np.einsum("slr,sLR->lLrR", M, M).reshape(D * D, D * D)
    w, vr = np.linalg.eig(T)
    R = np.real(vr[:, np.argmax(abs(w))]).reshape(D, D)
    w2, vl = np.linalg.eig(T.T)
    L = np.real(vl[:, np.argmax(abs(w2))]).reshape(D, D)
    h = W.heisenberg_bond_rotated()
    rho2 = np.einsum("lL,alm,bmr,cLn,dnR,rR->abcd", L, M, M, M, M, R).reshape(4, 4)
    eH = np.trace(rho2 @ h) / np.trace(rho2)
    rho1 = np.einsum("lL,alr,cLR,rR->ac", L, M, M, R)
    rho1 /= np.trace(rho1)
    eV = np.trace(np.kron(rho1, rho1) @ h)
    E, _ = evaluate([A], 1, 1, 8, 30, W.heisenberg_terms_rotated(), env0=_env0(1, 1, D, 8), grad=False)
    assert abs(E - (eH + eV)) < 1e-9


def test_trivial_boundary_is_a_fixed_point_of_the_nested_iteration():
    rng = np.random.default_rng(5)
    A = torch.tensor(np.abs(rng.standard_normal((2, 2, 2, 2, 2))))
    sp = []
    ctmrg(nested_cell([A], 1, 1), 8, 2, env=None, spectra_log=sp)
    for it in sp:
        for s in it:
            assert float(s[1:].abs().max()) < 1e-15


# ----------------------------------------------------------------------------- single vs double
@pytest.mark.parametrize("Lx,Ly", [(1, 1), (2, 2)])
@pytest.mark.parametrize("cutoff,tol", [(1e-5, 1e-5), (1e-10, 1e-7)])
def test_single_and_double_layer_agree(Lx, Ly, cutoff, tol, monkeypatch):
    # Appendix: nested and reduced contraction agree once chi is large enough;
    # what is left is the truncation of the spectra at the cutoff.
    import oracle.ctmrg as oc
    monkeypatch.setattr(oc, "CUTOFF", cutoff)
    rng = np.random.default_rng(7)
    D, chi = 2, 16
    As = [rng.random((2, D, D, D, D)) + 0.1 for _ in range(Lx * Ly)]
    h = W.heisenberg_bond()
    terms = [W.Term(x, y, k, 1.0, h) for y in range(Ly) for x in range(Lx) for k in (W.BOND_H, W.BOND_V)]
    En, _ = evaluate(As, Lx, Ly, chi, 20, terms, env0=_env0(Lx, Ly, D, chi), grad=False)
    Ed, _ = evaluate(As, Lx, Ly, chi, 20, terms, env0=None, grad=False, layer="double")
    assert abs(En - Ed) < tol


# ----------------------------------------------------------------------------- adjoint and gradient
@pytest.mark.parametrize("shape", [(12, 8, 4), (8, 12, 4), (10, 10, 5)])
def test_projector_adjoint_matches_autograd_of_plain_qr_svd(shape):
    torch.manual_seed(0)
    nr, nl, chi = shape
    N = torch.randn(nr, nl, dtype=DT, requires_grad=True)
    S = torch.randn(nr, nl, dtype=DT, requires_grad=True)
    wP, wQ = torch.randn(nl, chi, dtype=DT), torch.randn(nl, chi, dtype=DT)
    P, Q = projectors(N, S, chi)
    g1 = torch.autograd.grad((P * wP).sum() + (Q * wQ).sum(), (N, S))
    P2, Q2 = projectors_plain(N, S, chi)
    sg = torch.sign((P * P2).sum(0)).detach()
    assert float((P - P2 * sg).abs().max()) < 1e-12
    g2 = torch.autograd.grad((P2 * sg * wP).sum() + (Q2 * sg * wQ).sum(), (N, S))
    for a, b in zip(g1, g2):
        assert float((a - b).norm() / b.norm()) < 1e-9


def test_projector_product_reproduces_truncated_density_matrix():
    torch.manual_seed(1)
    N = torch.randn(12, 8, dtype=DT)
    S = torch.randn(12, 8, dtype=DT)
    P, Q = projectors(N, S, 3)
    U, s, Vh = torch.linalg.svd(N @ S.T)
    assert float((N @ P @ Q.T @ S.T - U[:, :3] @ torch.diag(s[:3]) @ Vh[:3]).abs().max()) < 1e-12


def test_gradient_matches_central_finite_differences():
    w = W.config("heis_d2_chi8")
    env0 = W.initial_environment(w)
    n_it = 8
    E, g = evaluate(w.tensors, 1, 1, w.chi, n_it, w.terms, env0=env0)
    A = w.tensors[0]
    rng = np.random.default_rng(1001)
    for _ in range(3):
        v = rng.standard_normal(A.shape)
        v /= np.linalg.norm(v)
        h = 1e-6 * np.linalg.norm(A)
        Ep, _ = evaluate([A + h * v], 1, 1, w.chi, n_it, w.terms, env0=env0, grad=False)
        Em, _ = evaluate([A - h * v], 1, 1, w.chi, n_it, w.terms, env0=env0, grad=False)
        fd = (Ep - Em) / (2 * h)
        # central differences at this step agree with smaller steps to ~1e-8 of |dE/dA| on these
        # inputs; the bar (relative to the gradient norm, v being a unit vector) sits above that
        # and well below the 1e-5 parity bar of the GPU gradient
        assert abs(fd - (g[0] * v).sum()) < 1e-6 * np.linalg.norm(g[0])


def test_scale_invariance_and_euler_relation():
    w = W.config("heis_d2_chi8")
    env0 = W.initial_environment(w)
    E1, g = evaluate(w.tensors, 1, 1, w.chi, 6, w.terms, env0=env0)
    E2, _ = evaluate([3.7 * w.tensors[0]], 1, 1, w.chi, 6, w.terms, env0=env0, grad=False)
    assert abs(E1 - E2) < 1e-12
    assert abs((g[0] * w.tensors[0]).sum()) < 1e-10 * np.abs(g[0]).sum()


def test_ring_array_roundtrip():
    w = W.config("ss_d6_chi64")
    w = W.Workload("s", 2, 2, 2, 2, 4, 0, [], [])
    arr = W.initial_environment(w)
    env = from_ring_arrays(arr, 4, 4)
    back = to_ring_arrays(env)
    assert all(np.array_equal(a, b) for s1, s2 in zip(arr, back) for a, b in zip(s1, s2))


# ----------------------------------------------------------------------------- symmetry invariants
def _bond_gauge(T, O, P):
    """Orthogonal gauge on the bonds: O on both horizontal legs (l, r), P on both vertical (u, d)."""
    T = np.einsum("sauvd,al,vr->slurd", T, O, O)
    return np.einsum("slurb,bd->slurd", np.einsum("slard,au->slurd", T, P), P)


def test_orthogonal_bond_gauge_leaves_energy_and_transforms_gradient():
    # A -> A with an orthogonal O on each bond leaves the PEPS unchanged (O O^t = 1 on every
    # contracted bond); once chi resolves the environment (chi=16 at D=2) the CTMRG energy agrees
    # to 1e-8 and the gradient transforms with the same O (measured 1.3e-9 and 2.9e-6)
    w = W.custom(1, 1, 2, 16, 30, seeds=[0], terms=W.heisenberg_terms_rotated())
    w.tensors = W.config("heis_d2_chi8").tensors
    A = w.tensors[0]
    env0 = W.initial_environment(w)
    rng = np.random.default_rng(21)
    O, _ = np.linalg.qr(rng.standard_normal((2, 2)))
    P, _ = np.linalg.qr(rng.standard_normal((2, 2)))
    E, g = evaluate([A], 1, 1, w.chi, w.n_iter, w.terms, env0=env0)
    E2, g2 = evaluate([_bond_gauge(A, O, P)], 1, 1, w.chi, w.n_iter, w.terms, env0=env0)
    assert abs(E - E2) < 1e-8
    assert np.linalg.norm(_bond_gauge(g[0], O, P) - g2[0]) < 3e-5 * np.linalg.norm(g2[0])


def test_c4v_symmetric_tensor_has_equal_bond_energies():
    # a tensor symmetrised over the square's rotations and reflections (legs l, u, r, d) with the
    # same Hamiltonian on both bonds: e_x = e_y up to the truncation (measured 1e-7 at chi=8)
    w = W.config("heis_d2_chi8")
    A = w.tensors[0]
    rot = lambda T: np.transpose(T, (0, 4, 1, 2, 3))   # (l,u,r,d) <- (d,l,u,r): 90 degrees
    refl = lambda T: np.transpose(T, (0, 3, 2, 1, 4))  # l <-> r
    S, X = np.zeros_like(A), A
    for _ in range(4):
        S, X = S + X + refl(X), rot(X)
    S /= 8
    pb = []
    evaluate([S], 1, 1, w.chi, 30, w.terms, env0=W.initial_environment(w), grad=False, per_bond=pb)
    assert len(pb) == 2
    assert abs(pb[0] - pb[1]) < 1e-6, pb


# ----------------------------------------------------------------------------- work counter
def test_multiply_add_counter_counts_contractions_and_decompositions():
    from oracle import counter
    counter.reset()
    a, b = torch.ones(3, 4, dtype=torch.float64), torch.ones(4, 5, dtype=torch.float64)
    counter.einsum("ij,jk->ik", a, b)
    assert counter.MACS["contraction"] == 3 * 4 * 5
    counter.einsum(a, [0, 1], b, [1, 2], [0, 2])
    assert counter.MACS["contraction"] == 2 * 60
    counter.reset()
    w = W.config("heis_d2_chi8")
    evaluate(w.tensors, 1, 1, w.chi, 1, w.terms, env0=W.initial_environment(w), grad=False)
    one = dict(counter.MACS)
    counter.reset()
    evaluate(w.tensors, 1, 1, w.chi, 2, w.terms, env0=W.initial_environment(w), grad=False)
    two = dict(counter.MACS)
    # the decompositions scale with the iterations exactly; contractions add one iteration's worth
    assert one["qr"] > 0 and one["svd"] > 0 and two["qr"] == 2 * one["qr"] and two["svd"] == 2 * one["svd"]
    assert two["contraction"] > one["contraction"]


# ----------------------------------------------------------------------------- convergence measure
def test_spectrum_change_by_hand_and_on_a_product_state():
    # delta = max over projector pairs of the largest entry-wise change of the normalised
    # truncated spectrum; worked by hand on two pairs of three values each.
    from oracle.ctmrg import spectrum_change
    prev = [torch.tensor([0.5, 0.3, 0.2], dtype=DT), torch.tensor([0.7, 0.2, 0.1], dtype=DT)]
    cur = [torch.tensor([0.6, 0.3, 0.1], dtype=DT), torch.tensor([0.65, 0.25, 0.1], dtype=DT)]
    assert abs(spectrum_change(prev, cur) - 0.1) < 1e-15
    assert abs(spectrum_change(cur, prev) - 0.1) < 1e-15
    assert spectrum_change(cur, cur) == 0.0
    # the logged spectra are s/sum(s): each sums to one, and a rank-one (D=1 product) state has
    # the spectrum (1, 0, ...) in every iteration, so delta is exactly zero from the start
    sp = []
    A = torch.tensor(W.product_site([0.6, 0.8]))
    ctmrg(nested_cell([A], 1, 1), 4, 3, env=from_ring_arrays(_env0(1, 1, 1, 4), 2, 2), spectra_log=sp)
    for it in sp:
        for s in it:
            assert abs(float(s.sum()) - 1.0) < 1e-14
    assert spectrum_change(sp[1], sp[2]) < 1e-15


def test_sign_mixed_random_tensors_do_not_converge_but_the_workload_inputs_do():
    # Why the workloads are not pure N(0, 1/(2 D^4)) draws: on such a tensor the nested CTMRG
    # with chi = 8 never settles -- the energy after n iterations jumps by O(1) from one n to the
    # next (one draw shown; D=4 and D=6, chi=64 behave the same) -- whereas the correlated core
    # plus eta = 0.2 Gaussian noise of the workloads converges.
    D, chi = 2, 8
    signed = np.random.default_rng(1).standard_normal((2, D, D, D, D)) / np.sqrt(2 * D**4)
    terms = W.heisenberg_terms_rotated()
    env0 = _env0(1, 1, D, chi)
    for A, lo, hi in ((signed, 0.1, np.inf), (W.noisy_ising_site(1, 2, D), 0.0, 1e-5)):
        Es = [evaluate([A], 1, 1, chi, n, terms, env0=env0, grad=False)[0] for n in (14, 16, 18, 20)]
        spread = max(Es) - min(Es)
        assert lo <= spread < hi, (Es, spread)


def test_gradient_does_not_depend_on_the_svd_algorithm_at_the_cutoff():
    # The pseudo-inverse cutoff is set where FP64 resolves every kept singular vector: there the
    # gradient is a property of the network, not of the SVD routine.  Two LAPACK drivers (QR
    # iteration and divide and conquer) must give the same energy and gradient well inside the
    # 1e-5 parity bar.  (At a cutoff of 1e-8 the same comparison differs by 4e-4.)
    import scipy.linalg
    import oracle.ctmrg as oc
    w = W.custom(2, 2, 2, 6, 3, seeds=[2, 3, 4, 5], terms=W.shastry_sutherland_terms(), name="ss_small")
    env0 = W.initial_environment(w)
    out = []
    orig = oc._svd
    try:
        for drv in ("gesvd", "gesdd"):
            def svd(M, drv=drv):
                U, s, Vh = scipy.linalg.svd(M.detach().numpy(), full_matrices=True, lapack_driver=drv)
                return torch.from_numpy(U), torch.from_numpy(s), torch.from_numpy(Vh.T.copy())
            oc._svd = svd
            out.append(evaluate(w.tensors, w.Lx, w.Ly, w.chi, w.n_iter, w.terms, env0=env0))
    finally:
        oc._svd = orig
    (E1, g1), (E2, g2) = out
    g1 = np.concatenate([x.ravel() for x in g1])
    g2 = np.concatenate([x.ravel() for x in g2])
    assert abs(E1 - E2) < 1e-12
    assert np.linalg.norm(g1 - g2) / np.linalg.norm(g1) < 1e-6


# ----------------------------------------------------------------------------- order parameters
def test_one_site_rdm_of_the_nested_cluster_equals_the_state_vector():
    # Eq. Mag1 needs one-site expectation values: the nested network with a single impurity Y,
    # contracted exactly on an open cluster, against <psi|S_a|psi>/<psi|psi> from the amplitudes
    from oracle.observables import SX, SZ, site_magnetization
    rng = np.random.default_rng(13)
    D, d, Lx, Ly = 2, 2, 3, 2
    sites = [[torch.tensor(rng.standard_normal((d, D, D, D, D))) for _ in range(Lx)] for _ in range(Ly)]
    psi = exact.state_vector(sites)
    for y in range(Ly):
        for x in range(Lx):
            m = site_magnetization(exact.nested_site_rdm(sites, (x, y), d))
            i = y * Lx + x
            assert abs(m[0] - exact.site_expectation_sv(psi, SX, i)) < 1e-12
            assert abs(m[2] - exact.site_expectation_sv(psi, SZ, i)) < 1e-12


def test_magnetization_of_product_neel_and_dimer_states():
    from oracle.observables import magnetization
    from oracle.ctmrg import ctmrg
    # D=1 product state: m = (v Sx v, 0, v Sz v) / |v|^2 exactly
    v = np.array([0.8, -0.45])
    A = torch.tensor(W.product_site(v))
    grid = nested_cell([A], 1, 1)
    env = ctmrg(grid, 4, 3, env=from_ring_arrays(_env0(1, 1, 1, 4), 2, 2))
    m, M = magnetization([A], 1, 1, env, grid)
    n2 = v @ v
    assert np.abs(m[0] - np.array([v[0] * v[1] / n2, 0.0, 0.5 * (v[0] ** 2 - v[1] ** 2) / n2])).max() < 1e-12
    assert abs(M - np.hypot(v[0] * v[1], 0.5 * (v[0] ** 2 - v[1] ** 2)) / n2) < 1e-12
    # rotated Neel state: full moment 1/2
    A = torch.tensor(W.neel_rotated_site())
    grid = nested_cell([A], 1, 1)
    env = ctmrg(grid, 4, 3, env=from_ring_arrays(_env0(1, 1, 1, 4), 2, 2))
    assert abs(magnetization([A], 1, 1, env, grid)[1] - 0.5) < 1e-12
    # dimer-singlet product state: every site is half of a singlet, so m_i = 0
    As = [torch.tensor(a) for a in W.dimer_singlet_sites()]
    grid = nested_cell(As, 2, 2)
    env = ctmrg(grid, 8, 4, env=from_ring_arrays(_env0(2, 2, 2, 8), 4, 4))
    m, M = magnetization(As, 2, 2, env, grid)
    assert np.abs(m).max() < 1e-12 and M < 1e-12


def test_plaquette_lists_are_the_empty_squares_of_the_cell():
    # geometry of Eq. Mag2: the two lists partition the 8 nearest-neighbour bonds, each list is the
    # boundary of one square, and neither square holds a J' dimer
    terms = W.shastry_sutherland_terms()
    a, b = W.shastry_sutherland_empty_plaquettes()
    assert sorted(a + b) == list(range(8))

    def square(px, py):
        want = {(px % 2, py % 2, W.BOND_H), (px % 2, (py + 1) % 2, W.BOND_H),
                (px % 2, py % 2, W.BOND_V), ((px + 1) % 2, py % 2, W.BOND_V)}
        return sorted(k for k, t in enumerate(terms[:8]) if (t.x, t.y, t.kind) in want)

    assert sorted(a) == square(1, 0) and sorted(b) == square(0, 1)
    dimers = [(t.x, t.y, t.kind) for t in terms if t.kind in (W.BOND_DIAG_DR, W.BOND_DIAG_UR)]
    assert dimers == [(0, 0, W.BOND_DIAG_DR), (1, 1, W.BOND_DIAG_UR)]   # inside squares (0,0), (1,1)


def test_plaquette_order_of_the_dimer_state_and_by_hand():
    from oracle.observables import plaquette_order
    a, b = W.shastry_sutherland_empty_plaquettes()
    vals = [0.1 * k for k in range(10)]
    assert abs(plaquette_order(vals, a, b) - 0.25 * abs(sum(vals[k] for k in a) - sum(vals[k] for k in b))) < 1e-15
    assert abs(plaquette_order(vals, a, b) - 0.25 * abs((0.2 + 0.6 + 0.3 + 0.1) - (0.4 + 0.0 + 0.5 + 0.7))) < 1e-15
    sites = W.dimer_singlet_sites()
    per = []
    evaluate(sites, 2, 2, 8, 4, W.shastry_sutherland_terms(), env0=_env0(2, 2, 2, 8), grad=False, per_bond=per)
    assert plaquette_order(per, a, b) < 1e-12


# ----------------------------------------------------------------------------- fixed-point gradient
@pytest.fixture(scope="module")
def _converged_d2():
    from oracle.fixed_point import converge
    w = W.config("heis_d2_chi8")
    env, n, res = converge(w.tensors, w.Lx, w.Ly, w.chi, W.initial_environment(w), tol=1e-13)
    assert res <= 1e-13
    return w, env


def test_sign_gauge_gives_an_elementwise_fixed_point(_converged_d2):
    # with the projector SVD's sign gauge fixed, one more iteration reproduces the converged
    # environment entry by entry (the premise of the fixed-point gradient)
    from oracle.api import warm_environment
    w, env = _converged_d2
    nxt = warm_environment(w.tensors, w.Lx, w.Ly, w.chi, 1, env)
    a = np.concatenate([x.ravel() for s in env for x in s])
    b = np.concatenate([x.ravel() for s in nxt for x in s])
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


def test_fixed_point_gradient_matches_finite_differences_of_the_converged_energy(_converged_d2):
    # E(A) = e(A, env*(A)): every perturbed state is re-converged from env* to 1e-13, so the
    # central difference is the derivative of the converged energy itself (not of a fixed
    # number of iterations)
    from oracle.fixed_point import converge, fixed_point_energy_grad
    w, env = _converged_d2
    E, g, n_adj, res = fixed_point_energy_grad(w.tensors, w.Lx, w.Ly, w.chi, w.terms, env)
    assert res <= 1e-12 and n_adj < 200
    A = w.tensors[0]
    h = 1e-5
    rng = np.random.default_rng(77)
    idx = rng.choice(A.size, size=4, replace=False)
    for k in idx:
        vals = []
        for sgn in (1, -1):
            Ap = A.copy().ravel()
            Ap[k] += sgn * h
            Ap = Ap.reshape(A.shape)
            envp, _, r = converge([Ap], w.Lx, w.Ly, w.chi, env, tol=1e-13, chunk=5)
            assert r <= 1e-13
            vals.append(evaluate([Ap], w.Lx, w.Ly, w.chi, 0, w.terms, env0=envp, grad=False)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[0].ravel()[k] - fd) <= 1e-6 * np.abs(g[0]).max(), (k, g[0].ravel()[k], fd)


def test_fixed_point_gradient_is_the_limit_of_the_unrolled_one(_converged_d2):
    # from the fixed point, the unrolled reverse mode over n iterations is the Neumann series cut
    # after n terms: it approaches the fixed-point gradient as n grows; Euler's relation holds
    from oracle.fixed_point import fixed_point_energy_grad
    w, env = _converged_d2
    E, g, _, _ = fixed_point_energy_grad(w.tensors, w.Lx, w.Ly, w.chi, w.terms, env)
    errs = []
    for n in (5, 40):
        Eu, gu = evaluate(w.tensors, w.Lx, w.Ly, w.chi, n, w.terms, env0=env)
        assert abs(Eu - E) <= 1e-13
        errs.append(np.linalg.norm(gu[0] - g[0]) / np.linalg.norm(g[0]))
    assert errs[1] <= 1e-7 and errs[1] < errs[0] / 100, errs
    assert abs(np.sum(g[0] * w.tensors[0])) <= 1e-10 * np.linalg.norm(g[0]) * np.linalg.norm(w.tensors[0])


# ----------------------------------------------------------------------------- warm-start network
def test_mlp_gradient_matches_central_differences_of_the_loss():
    from oracle import mlp
    rng = np.random.default_rng(5)
    dims = [7, 6, 5, 4]
    W = [rng.standard_normal((dims[k + 1], dims[k])) / 2 for k in range(3)]
    b = [rng.standard_normal(dims[k + 1]) / 2 for k in range(3)]
    x = rng.standard_normal((3, 7))
    t = rng.standard_normal((3, 4))
    L, dW, db = mlp.loss_and_grad(x, t, W, b)
    h = 1e-6
    for k in range(3):
        for (i, j) in ((0, 0), (dims[k + 1] - 1, dims[k] - 1), (1, 2)):
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[k][i, j] += h
            Wm[k][i, j] -= h
            fd = (mlp.loss_and_grad(x, t, Wp, b)[0] - mlp.loss_and_grad(x, t, Wm, b)[0]) / (2 * h)
            assert abs(dW[k][i, j] - fd) <= 1e-8 * max(1.0, abs(fd)), (k, i, j)
        bp = [v.copy() for v in b]
        bm = [v.copy() for v in b]
        bp[k][1] += h
        bm[k][1] -= h
        fd = (mlp.loss_and_grad(x, t, W, bp)[0] - mlp.loss_and_grad(x, t, W, bm)[0]) / (2 * h)
        assert abs(db[k][1] - fd) <= 1e-8 * max(1.0, abs(fd))


def test_gelu_derivative_and_adam_first_step():
    from oracle import mlp
    z = np.linspace(-4, 4, 17)
    h = 1e-6
    assert np.allclose(mlp.gelu_prime(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-9)
    assert np.allclose(mlp.gelu(np.array([0.0, 10.0, -10.0])), [0.0, 10.0, 0.0], atol=1e-12)
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 0.01, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
