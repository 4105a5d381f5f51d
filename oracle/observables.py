"""Order parameters of the Results section from a CTMRG environment (oracle, FP64).

Test infrastructure only: the product path computes these in libctm (ctm_magnetization,
ctm_plaquette_order).

* Eq. Mag1: M = (1/N) sum_i |m_i|, m_i = (<S_x>, <S_y>, <S_z>) on the N inequivalent sites of the
  unit cell.  The one-site reduced density matrix of PEPS site (x, y) is the nested block
  [A Y; X A*] with the physical line of its Y cut open (the impurity tensor of Sec. NTN), closed by
  the environment.  With real tensors Tr(rho S_y) is purely imaginary and <S_y>, its real part,
  vanishes.  A sublattice rotation flips S_x and S_z of one sublattice and leaves |m_i| unchanged.
* Eq. Mag2: M_p = (1/4) |sum_{<ij> in A} <S_i.S_j> - sum_{<ij> in B} <S_i.S_j>| over the
  nearest-neighbour bonds of the two inequivalent empty plaquettes A and B; the bond values are
  the per-bond Tr(rho h)/Tr(rho) of the energy estimator.

Parity: pinned by tests/test_oracle_pins.py (exact finite cluster, D=1 product states, the Neel
and the dimer-singlet states).
"""
from __future__ import annotations

import numpy as np
import torch

from .energy import block_rdm
from .nested import DT, nested_cell, y_impurity

SX = np.array([[0.0, 0.5], [0.5, 0.0]])
SZ = np.array([[0.5, 0.0], [0.0, -0.5]])


def site_rdm(As, Lx, Ly, env, x, y, grid=None):
    """One-site RDM [ket sigma][bra sigma'] of PEPS site (x, y) from the nested network."""
    d, D = As[0].shape[0], As[0].shape[1]
    if grid is None:
        grid = nested_cell(As, Lx, Ly)
    t, ls = block_rdm(grid, env, 2 * y, 2 * x, 2, 2, {(0, 1): (y_impurity(D, d), "k", "b")})
    return t.permute(ls.index("k"), ls.index("b"))


def site_magnetization(rho):
    """(<S_x>, <S_y>, <S_z>) of a 2 x 2 one-site RDM (<S_y> = 0 for real tensors)."""
    r = torch.as_tensor(rho, dtype=DT)
    tr = torch.trace(r)
    sx = float(torch.einsum("ab,ba->", r, torch.as_tensor(SX)) / tr)
    sz = float(torch.einsum("ab,ba->", r, torch.as_tensor(SZ)) / tr)
    return np.array([sx, 0.0, sz])


def magnetization(As, Lx, Ly, env, grid=None):
    """Eq. Mag1: (per-site m as an (Lx*Ly, 3) array, M)."""
    m = np.stack([site_magnetization(site_rdm(As, Lx, Ly, env, x, y, grid))
                  for y in range(Ly) for x in range(Lx)])
    return m, float(np.linalg.norm(m, axis=1).mean())


def plaquette_order(bond_values, terms_a, terms_b):
    """Eq. Mag2 from per-term bond values (<S_i.S_j> for Heisenberg bonds)."""
    return 0.25 * abs(sum(bond_values[k] for k in terms_a) - sum(bond_values[k] for k in terms_b))
