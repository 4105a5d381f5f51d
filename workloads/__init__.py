"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the method: it only draws site tensors,
writes down the spin-1/2 bond operators of the two lattice models, and lists
the bond terms of each workload.  Both the oracle (``oracle/``) and the CUDA
path read their inputs from here, so that the two sides see identical data.

Conventions
-----------
* A site tensor is a float64 array ``A[s, l, u, r, d]`` (physical index first,
  then the four virtual legs left, up, right, down), row-major.
* PEPS site ``(x, y)`` of an ``Lx x Ly`` unit cell (x to the right, y down) is
  stored at index ``y * Lx + x``.
* A bond operator ``h`` is a real ``d^2 x d^2`` matrix, row index
  ``s1 * d + s2`` and column index ``s1' * d + s2'``, where site 1 is the
  first site of the bond (left, top, or as listed for the diagonal kinds).
* Bond kinds (both endpoints given relative to ``(x, y)``):
  ``H``: (x, y)-(x+1, y); ``V``: (x, y)-(x, y+1);
  ``DIAG_DR``: (x, y)-(x+1, y+1); ``DIAG_UR``: (x+1, y)-(x, y+1).
"""
from __future__ import annotations

import dataclasses
import numpy as np

BOND_H, BOND_V, BOND_DIAG_DR, BOND_DIAG_UR = 0, 1, 2, 3
BOND_NAMES = {BOND_H: "H", BOND_V: "V", BOND_DIAG_DR: "DIAG_DR", BOND_DIAG_UR: "DIAG_UR"}

# ---------------------------------------------------------------- spin-1/2 operators
SZ = np.array([[0.5, 0.0], [0.0, -0.5]])
SP = np.array([[0.0, 1.0], [0.0, 0.0]])  # S^+ |down> = |up>, basis (up, down)
SM = SP.T.copy()


def heisenberg_bond() -> np.ndarray:
    """S_1 . S_2 = Sz Sz + (S+ S- + S- S+)/2 as a 4x4 real matrix (Eq. SSM, one term)."""
    return np.kron(SZ, SZ) + 0.5 * (np.kron(SP, SM) + np.kron(SM, SP))


def heisenberg_bond_rotated() -> np.ndarray:
    """S_1 . S_2 after the sublattice rotation U = -i sigma_y on site 2.

    -i sigma_y = [[0, -1], [1, 0]] is real; conjugating site 2 by it maps
    (Sx, Sy, Sz) -> (-Sx, Sy, -Sz), so the bond becomes
    -Sz Sz - (S+ S+ + S- S-)/2.  This is the input of the 1-site ansatz
    (Sec. Outlook, local spin rotation on one sublattice).
    """
    U = np.array([[0.0, -1.0], [1.0, 0.0]])
    W = np.kron(np.eye(2), U)
    return W.T @ heisenberg_bond() @ W


@dataclasses.dataclass
class Term:
    x: int
    y: int
    kind: int
    coupling: float
    h: np.ndarray  # d^2 x d^2


@dataclasses.dataclass
class Workload:
    name: str
    Lx: int
    Ly: int
    d: int
    D: int
    chi: int
    n_iter: int
    tensors: list  # Lx*Ly arrays [d, D, D, D, D], float64
    terms: list    # list[Term]
    precision: str = "fp64"

    @property
    def n_sites(self) -> int:
        return self.Lx * self.Ly


ISING_K = 0.42       # amplitude coupling; the norm network is the Ising model at 2*(K/2)*2 = K, K_c = 0.4407
ISING_NOISE = 0.05


def ising_site(seed: int, d: int, D: int, K: float = ISING_K, noise: float = ISING_NOISE) -> np.ndarray:
    """Sign-free correlated PEPS tensor: the Ising wave function plus positive noise.

    psi(s) = prod_<ij> exp(K s_i s_j / 2) (s = +-1 for sigma = up, down) is a
    D=2 PEPS with A[s; l, u, r, d] = W[s,l] W[s,u] W[s,r] W[s,d], where
    W W^t = exp(K s s' / 2).  Its norm network is the classical Ising model at
    coupling K, close to criticality for K = 0.42, so the environment spectra
    decay slowly.  The tensor is embedded in bond dimension D and every entry
    gets noise * |N(0,1)| from ``np.random.default_rng(seed)``; the result is
    scaled to max-abs 1.
    """
    assert d == 2
    spin = np.array([1.0, -1.0])
    B = np.exp(0.5 * K * np.outer(spin, spin))
    w, v = np.linalg.eigh(B)
    Wm = v @ np.diag(np.sqrt(w)) @ v.T
    A = np.zeros((d, D, D, D, D))
    k = min(2, D)
    core = np.einsum("sl,su,sr,sd->slurd", Wm[:, :k], Wm[:, :k], Wm[:, :k], Wm[:, :k])
    A[:, :k, :k, :k, :k] = core
    A += noise * np.abs(np.random.default_rng(seed).standard_normal(A.shape))
    return A / np.abs(A).max()


NOISE_ETA = 0.15    # amplitude of the sign-mixed Gaussian part of the workload tensors


def noisy_ising_site(seed: int, d: int, D: int, eta: float = NOISE_ETA, K: float = ISING_K) -> np.ndarray:
    """Random-normal site tensor around a correlated sign-free core.

    The Ising wave function at coupling K (``ising_site`` without noise, scaled to max-abs 1)
    occupies the first two states of every bond; every entry of the D-dimensional tensor then
    gets eta * N(0, 1) from ``np.random.default_rng(seed)`` (signs mixed), and the result is
    scaled to max-abs 1.  With eta = 0.15 every bond state carries weight: at D=6, chi=64 the
    bond density matrices of the nested CTMRG are numerically of full rank (about 380 of 384
    singular values above 1e-13 s_1), all 64 kept values lie above 7e-6 s_1 once converged,
    and the iteration converges (spectrum change 5e-6 after 50 iterations).  Pure
    N(0, sigma^2) draws (eta -> infinity), and eta >= 0.25 at D=6, make the fixed-iteration
    function chaotic: the energy jumps by O(1) from one iteration to the next
    (tests/test_oracle_pins.py shows it at D=2).
    """
    A = ising_site(seed, d, D, K=K, noise=0.0)
    A = A / np.abs(A).max()
    A = A + eta * np.random.default_rng(seed).standard_normal(A.shape)
    return A / np.abs(A).max()


def random_site(seed: int, d: int, D: int, std: float | None = None, maxabs: bool = False,
                signed: bool = False) -> np.ndarray:
    """|N(0,1)| draw from ``np.random.default_rng(seed)``, scaled by ``std`` or to max-abs 1.

    The absolute value is taken because the nested single-layer CTMRG does not
    converge on sign-mixed random tensors (its cuts are not Hermitian; the
    iteration is then chaotic), while the sublattice-rotated Heisenberg ground
    state it is meant for is sign-free.  ``signed=True`` keeps the raw draw.
    """
    a = np.random.default_rng(seed).standard_normal((d, D, D, D, D))
    if not signed:
        a = np.abs(a)
    if maxabs:
        a = a / np.abs(a).max()
    elif std is not None:
        a = a * std
    return a


def heisenberg_terms_rotated(J: float = 1.0) -> list:
    """1-site ansatz with sublattice rotation: one H and one V bond per site."""
    h = heisenberg_bond_rotated()
    return [Term(0, 0, BOND_H, J, h), Term(0, 0, BOND_V, J, h)]


def shastry_sutherland_terms(J: float = 0.7, Jp: float = 1.0) -> list:
    """Shastry-Sutherland model on a 2x2 cell [A B; C F] (Eq. SSM).

    J on every nearest-neighbour bond (8 per cell), J' on the two dimer
    diagonals per cell: A(0,0)-F(1,1) and B(1,0)-C(0,1) of the next cell up
    and to the right, i.e. the DIAG_UR bond of the plaquette whose upper-left
    site is (1, 1).
    """
    h = heisenberg_bond()
    terms = []
    for y in range(2):
        for x in range(2):
            terms.append(Term(x, y, BOND_H, J, h))
            terms.append(Term(x, y, BOND_V, J, h))
    terms.append(Term(0, 0, BOND_DIAG_DR, Jp, h))
    terms.append(Term(1, 1, BOND_DIAG_UR, Jp, h))
    return terms


def shastry_sutherland_empty_plaquettes():
    """Term indices (into ``shastry_sutherland_terms()``) of the two inequivalent empty plaquettes.

    The squares of the 2x2 cell [A B; C F] are labelled by their upper-left site.  The squares at
    (0, 0) and (1, 1) hold the J' dimers (A-F, and B-C of the neighbouring cells); the squares at
    (1, 0) and (0, 1) are empty.  Square (px, py) has the bonds H(px, py), H(px, py+1), V(px, py)
    and V(px+1, py), coordinates mod 2; with the term order H(x,y), V(x,y) for y, x in 0, 1:
      square (1, 0): H(1,0)=2, H(1,1)=6, V(1,0)=3, V(0,0)=1
      square (0, 1): H(0,1)=4, H(0,0)=0, V(0,1)=5, V(1,1)=7
    """
    return [2, 6, 3, 1], [4, 0, 5, 7]


def config(name: str) -> Workload:
    """The seeded workloads: shapes of the paper's runs, random-normal tensors around a correlated core.

    heis_d2_chi8:  rotated Heisenberg, 1-site, D=2, chi=8, 20 iterations, seed 0
    heis_d4_chi32: rotated Heisenberg, 1-site, D=4, chi=32, 40 iterations, seed 1
    ss_d6_chi64:   Shastry-Sutherland J=0.7, J'=1, 2x2 cell, D=6, chi=64,
                   50 iterations, seeds 2..5 (one per site)
    heis_d9_chi81: rotated Heisenberg, 1-site, D=9, chi=81, 60 iterations, seed 6
    Every site tensor is ``noisy_ising_site(seed, 2, D)``.
    """
    d = 2
    if name == "heis_d2_chi8":
        return Workload(name, 1, 1, d, 2, 8, 20, [noisy_ising_site(0, d, 2)], heisenberg_terms_rotated())
    if name == "heis_d4_chi32":
        return Workload(name, 1, 1, d, 4, 32, 40, [noisy_ising_site(1, d, 4)], heisenberg_terms_rotated(),
                        precision="tf32")
    if name == "ss_d6_chi64":
        ts = [noisy_ising_site(s, d, 6) for s in (2, 3, 4, 5)]
        return Workload(name, 2, 2, d, 6, 64, 50, ts, shastry_sutherland_terms(), precision="bf16")
    if name == "heis_d9_chi81":
        return Workload(name, 1, 1, d, 9, 81, 60, [noisy_ising_site(6, d, 9)], heisenberg_terms_rotated(),
                        precision="bf16")
    raise KeyError(name)


def custom(Lx, Ly, D, chi, n_iter, seeds, terms, d=2, name="custom") -> Workload:
    """A workload of arbitrary size drawn the same way (used by scaled-down tests)."""
    ts = [noisy_ising_site(s, d, D) for s in seeds]
    assert len(ts) == Lx * Ly
    return Workload(name, Lx, Ly, d, D, chi, n_iter, ts, terms)


# --------------------------------------------------------------- special product states
def neel_rotated_site(D: int = 1, d: int = 2) -> np.ndarray:
    """D=1 rotated Neel state: A[s] = delta_{s, up} (ferromagnet after rotation)."""
    a = np.zeros((d, D, D, D, D))
    a[0, 0, 0, 0, 0] = 1.0
    return a


def product_site(v) -> np.ndarray:
    """D=1 product state A[s] = v_s."""
    v = np.asarray(v, dtype=np.float64)
    return v.reshape(-1, 1, 1, 1, 1).copy()


def dimer_singlet_sites() -> list:
    """Exact D=2 PEPS of the Shastry-Sutherland dimer-singlet product state.

    Cell [A B; C F].  Every J' singlet is routed along an L-shaped path through
    one intermediate site; unused virtual legs carry index 0.  With the
    singlet matrix eps = [[0, 1], [-1, 0]] / sqrt(2):
      A[s; l, u, d] = delta_{l u} delta_{s d}      (r = 0)
      B[s; r]       = delta_{s r}                  (l = u = d = 0)
      C[s; u, r, d] = delta_{u r} eps_{d s}        (l = 0)
      F[s; l]       = eps_{l s}                    (u = r = d = 0)
    The A-F singlet runs A -down-> C -right-> F; the B-C' singlet (C' in the
    cell up and to the right) runs B -right-> A' -up-> C'.
    """
    D, d = 2, 2
    eps = np.array([[0.0, 1.0], [-1.0, 0.0]]) / np.sqrt(2.0)
    A = np.zeros((d, D, D, D, D))
    B = np.zeros((d, D, D, D, D))
    C = np.zeros((d, D, D, D, D))
    F = np.zeros((d, D, D, D, D))
    for s in range(d):
        for k in range(D):
            A[s, k, k, 0, s] = 1.0          # l = u = k, d = s
            B[s, 0, 0, s, 0] = 1.0          # r = s
            for t in range(D):
                C[s, 0, k, k, t] = eps[t, s]  # u = r = k, d = t
            F[s, k, 0, 0, 0] = eps[k, s]    # l = k
    return [A, B, C, F]


# --------------------------------------------------------------- nested layout and initial environment
ENV_SLOTS = ("C_ul", "T_u", "C_ur", "T_r", "C_dr", "T_d", "C_dl", "T_l")


def nested_leg_dims(i: int, j: int, D: int, d: int):
    """(left, up, right, down) bond dimensions of nested site (row i, col j).

    Ket at (even, even): right leg fused with sigma (D d).  Y at (even, odd):
    left and down legs D d.  X at (odd, even): all D.  Bra at (odd, odd): up
    leg fused with sigma (D d).
    """
    Dd = D * d
    if i % 2 == 0 and j % 2 == 0:
        return (D, D, Dd, D)
    if i % 2 == 0:
        return (Dd, D, D, Dd)
    if j % 2 == 0:
        return (D, D, D, D)
    return (D, Dd, D, D)


def env_shapes(Lx: int, Ly: int, D: int, d: int, chi: int):
    """Shapes of the 8 environment tensors of every nested site, row-major over the
    2Ly x 2Lx nested cell.  Ring convention (clockwise around the site):
    C: [prev, next], T: [prev, in, next], slots in ENV_SLOTS order, where
    C_ul = [down, right], T_u = [left, in, right], C_ur = [left, down],
    T_r = [up, in, down], C_dr = [up, left], T_d = [right, in, left],
    C_dl = [right, up], T_l = [down, in, up]."""
    out = []
    for i in range(2 * Ly):
        for j in range(2 * Lx):
            l, u, r, dn = nested_leg_dims(i, j, D, d)
            out.append([(chi, chi), (chi, u, chi), (chi, chi), (chi, r, chi),
                        (chi, chi), (chi, dn, chi), (chi, chi), (chi, l, chi)])
    return out


def initial_environment(w, seed: int = 12345):
    """Seeded positive random initial environment: every entry U(0,1).

    Drawn site by site (row-major), slot by slot (ENV_SLOTS order), each
    array in C order, from one ``np.random.default_rng(seed)`` stream.
    """
    rng = np.random.default_rng(seed)
    return [[rng.random(shp) for shp in site] for site in env_shapes(w.Lx, w.Ly, w.D, w.d, w.chi)]
