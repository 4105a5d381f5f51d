"""Nested single-layer network and reduced double-layer tensor (oracle, FP64).

Sec. NTN: instead of summing the physical index sigma into the reduced tensor
T^a (Eq. Tred, bond D^2), the nested network keeps the ket A and the bra A* as
separate sites of one square lattice.  Virtual tensors sit where ket and bra
lines cross (Eq. XY):

    X_{ijkl} = delta_ij delta_kl,   Y_{i sigma, j, k, l sigma'} = delta_ij delta_kl delta_{sigma sigma'}.

Readings (the figure that fixes the wiring is missing from the text):

* Leg order of every nested site is (left, up, right, down).
* Per PEPS site the nested cell is [A  Y; X  A*]: ket at (even row, even col),
  Y at (even, odd), X at (odd, even), bra at (odd, odd).  Rows grow downward.
* Y passes the ket horizontal line left->right and the bra vertical line
  up->down, and carries sigma from A's right leg to A*'s up leg.  So
  Y.left = (i, sigma) and Y.down = (l, sigma') have dimension D d, as the
  footnote on bond dimensions states; every other bond has dimension D.
* Fused legs put the virtual index first: (r, sigma) -> r * d + sigma.
* Real tensors only, so A* = A.

Parity: pinned by the finite-cluster tests (exact state vector vs. nested and
double-layer contraction, ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import torch

from .counter import einsum as counted_einsum

DT = torch.float64
KET, YSITE, XSITE, BRA = "A", "Y", "X", "A*"


def site_kind(i: int, j: int) -> str:
    """Kind of nested site (row i, col j)."""
    if i % 2 == 0:
        return KET if j % 2 == 0 else YSITE
    return XSITE if j % 2 == 0 else BRA


def ket_tensor(A: torch.Tensor) -> torch.Tensor:
    """a[l, u, (r, s), d] from A[s, l, u, r, d]."""
    d, D = A.shape[0], A.shape[1]
    return A.permute(1, 2, 3, 0, 4).reshape(D, D, D * d, D)


def bra_tensor(A: torch.Tensor) -> torch.Tensor:
    """a*[l, (u, s), r, d] from A[s, l, u, r, d] (real: A* = A)."""
    d, D = A.shape[0], A.shape[1]
    return A.permute(1, 2, 0, 3, 4).reshape(D, D * d, D, D)


def x_tensor(D: int) -> torch.Tensor:
    """X[l, u, r, d] = delta_lr delta_ud."""
    eye = torch.eye(D, dtype=DT)
    return counted_einsum("lr,ud->lurd", eye, eye)


def y_tensor(D: int, d: int) -> torch.Tensor:
    """Y[(i, s), k, j, (l, s')] = delta_ij delta_kl delta_ss'   (legs left, up, right, down)."""
    eD, ed = torch.eye(D, dtype=DT), torch.eye(d, dtype=DT)
    y = counted_einsum("ij,kl,st->iskjlt", eD, eD, ed)
    return y.reshape(D * d, D, D, D * d)


def y_impurity(D: int, d: int) -> torch.Tensor:
    """Y with the sigma line cut open: Y[(i,s), k, j, (l,s'), a, b] = delta_ij delta_kl delta_sa delta_s'b.

    Leg ``a`` is the ket's physical index and leg ``b`` the bra's; the impurity
    tensors of the local energy terms (Sec. NTN, last paragraph).
    """
    eD, ed = torch.eye(D, dtype=DT), torch.eye(d, dtype=DT)
    y = counted_einsum("ij,kl,sa,tb->iskjltab", eD, eD, ed, ed)
    return y.reshape(D * d, D, D, D * d, d, d)


def nested_cell(As: list, Lx: int, Ly: int) -> list:
    """2Ly x 2Lx grid of nested site tensors (rank 4) for PEPS tensors As[y*Lx+x]."""
    d, D = As[0].shape[0], As[0].shape[1]
    X, Y = x_tensor(D), y_tensor(D, d)
    grid = []
    for i in range(2 * Ly):
        row = []
        for j in range(2 * Lx):
            p = (i // 2) * Lx + (j // 2)
            k = site_kind(i, j)
            row.append({KET: lambda: ket_tensor(As[p]), BRA: lambda: bra_tensor(As[p]),
                        XSITE: lambda: X, YSITE: lambda: Y}[k]())
        grid.append(row)
    return grid


def reduced_tensor(A: torch.Tensor) -> torch.Tensor:
    """Double-layer T^a[(l l'), (u u'), (r r'), (d d')] = sum_s A[s..] A[s..]  (Eq. Tred)."""
    D = A.shape[1]
    T = counted_einsum("slurd,sLURD->lLuUrRdD", A, A)
    return T.reshape(D * D, D * D, D * D, D * D)


def reduced_impurity(A: torch.Tensor) -> torch.Tensor:
    """T^a with the physical index left open: [..., a, b], a = ket sigma, b = bra sigma."""
    D = A.shape[1]
    T = counted_einsum("alurd,bLURD->lLuUrRdDab", A, A)
    d = A.shape[0]
    return T.reshape(D * D, D * D, D * D, D * D, d, d)


def double_cell(As: list, Lx: int, Ly: int) -> list:
    """Ly x Lx grid of reduced tensors."""
    return [[reduced_tensor(As[y * Lx + x]) for x in range(Lx)] for y in range(Ly)]
