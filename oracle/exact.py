"""Finite clusters contracted without any truncation (oracle, FP64).

Used to pin the nested wiring, the impurity tensors, the bond operators and
the energy normalisation independently of CTMRG:

* ``state_vector``   - the PEPS of an open Lx x Ly cluster (every virtual leg
                        leaving the cluster fixed to index 0) contracted into
                        its 2^N amplitudes.
* ``bond_expectation_sv`` - <psi|h_b|psi>/<psi|psi> straight from the amplitudes.
* ``nested_bond_rdm`` / ``double_bond_rdm`` - the same two-site RDM from the
                        nested single-layer network (Eq. XY with the impurity
                        Y) and from the reduced double-layer network (Eq. Tred),
                        contracted exactly.
* ``nested_site_rdm`` / ``site_expectation_sv`` - a one-site RDM of the nested network
                        (one impurity Y) and the one-site expectation value from the amplitudes.
* ``lanczos_ground``  - the exact ground energy of the cluster Hamiltonian.

Parity: these are definitions written out; pinned against each other and
against the variational bound in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .energy import contract_pair
from .nested import (DT, bra_tensor, ket_tensor, reduced_impurity, reduced_tensor, site_kind,
                     x_tensor, y_impurity, y_tensor)


def _contract_sequence(items):
    acc = items[0]
    for it in items[1:]:
        acc = contract_pair(acc, it)
    return acc


def _fix_outer(t, ls, top, left, bottom, right):
    """Fix the outer legs among (l, u, r, d) -- the first four axes -- to index 0 and drop them."""
    fixed = [left, top, right, bottom]
    for ax in (3, 2, 1, 0):
        if fixed[ax]:
            t = t.select(ax, 0)
    return t, [l for ax, l in enumerate(ls) if ax >= 4 or not fixed[ax]]


def state_vector(sites):
    """sites[y][x] = A[s, l, u, r, d]; returns psi with one axis per site, row-major."""
    Ly, Lx = len(sites), len(sites[0])
    items = []
    for y in range(Ly):
        for x in range(Lx):
            A = sites[y][x].permute(1, 2, 3, 4, 0)            # [l, u, r, d, s]
            ls = [("h", y, x - 1), ("v", y - 1, x), ("h", y, x), ("v", y, x), ("s", y, x)]
            items.append(_fix_outer(A, ls, y == 0, x == 0, y == Ly - 1, x == Lx - 1))
    t, ls = _contract_sequence(items)
    keep = [ls.index(("s", y, x)) for y in range(Ly) for x in range(Lx)]
    return t.permute(*keep)


def _apply_bond(psi, h, i, j):
    d = psi.shape[0]
    n = psi.dim()
    perm = [i, j] + [k for k in range(n) if k not in (i, j)]
    t = psi.permute(*perm).reshape(d * d, -1)
    t = (torch.as_tensor(h, dtype=DT) @ t).reshape([d, d] + [d] * (n - 2))
    inv = np.argsort(perm).tolist()
    return t.permute(*inv)


def bond_expectation_sv(psi, h, i, j):
    hpsi = _apply_bond(psi, h, i, j)
    return float((psi * hpsi).sum() / (psi * psi).sum())


def cluster_bonds(Lx, Ly):
    """Nearest-neighbour bonds of an open cluster as ((x1,y1),(x2,y2)) pairs."""
    b = []
    for y in range(Ly):
        for x in range(Lx):
            if x + 1 < Lx:
                b.append(((x, y), (x + 1, y)))
            if y + 1 < Ly:
                b.append(((x, y), (x, y + 1)))
    return b


def nested_bond_rdm(sites, s1, s2, d):
    """Exact two-site RDM of sites s1=(x,y), s2 from the nested network of the open cluster."""
    Ly, Lx = len(sites), len(sites[0])
    D = sites[0][0].shape[1]
    X, Y, Yi = x_tensor(D), y_tensor(D, d), y_impurity(D, d)
    R, C = 2 * Ly, 2 * Lx
    imp = {(2 * s1[1], 2 * s1[0] + 1): ("k1", "b1"), (2 * s2[1], 2 * s2[0] + 1): ("k2", "b2")}
    items = []
    for i in range(R):
        for j in range(C):
            k = site_kind(i, j)
            p = sites[i // 2][j // 2]
            extra = []
            if k == "A":
                t = ket_tensor(p)
            elif k == "A*":
                t = bra_tensor(p)
            elif k == "X":
                t = X
            elif (i, j) in imp:
                t = Yi
                extra = list(imp[(i, j)])
            else:
                t = Y
            ls = [("h", i, j - 1), ("v", i - 1, j), ("h", i, j), ("v", i, j)] + extra
            items.append(_fix_outer(t, ls, i == 0, j == 0, i == R - 1, j == C - 1))
    t, ls = _contract_sequence(items)
    order = [ls.index(l) for l in ("k1", "k2", "b1", "b2")]
    return t.permute(*order).reshape(d * d, d * d)


def nested_site_rdm(sites, s, d):
    """Exact one-site RDM [ket sigma][bra sigma'] of site s=(x,y) from the nested network of the open
    cluster: the Y of that site carries its physical line cut open (Sec. NTN impurity)."""
    Ly, Lx = len(sites), len(sites[0])
    D = sites[0][0].shape[1]
    X, Y, Yi = x_tensor(D), y_tensor(D, d), y_impurity(D, d)
    R, C = 2 * Ly, 2 * Lx
    items = []
    for i in range(R):
        for j in range(C):
            k = site_kind(i, j)
            p = sites[i // 2][j // 2]
            extra = []
            if k == "A":
                t = ket_tensor(p)
            elif k == "A*":
                t = bra_tensor(p)
            elif k == "X":
                t = X
            elif (i, j) == (2 * s[1], 2 * s[0] + 1):
                t = Yi
                extra = ["k", "b"]
            else:
                t = Y
            ls = [("h", i, j - 1), ("v", i - 1, j), ("h", i, j), ("v", i, j)] + extra
            items.append(_fix_outer(t, ls, i == 0, j == 0, i == R - 1, j == C - 1))
    t, ls = _contract_sequence(items)
    return t.permute(ls.index("k"), ls.index("b"))


def site_expectation_sv(psi, op, i):
    """<psi|op_i|psi>/<psi|psi> for a one-site operator op (d x d) on site i."""
    n = psi.dim()
    perm = [i] + [k for k in range(n) if k != i]
    t = psi.permute(*perm).reshape(psi.shape[i], -1)
    return float((t * (torch.as_tensor(op, dtype=DT) @ t)).sum() / (psi * psi).sum())


def double_bond_rdm(sites, s1, s2, d):
    """Exact two-site RDM from the reduced (double-layer) network of the open cluster."""
    Ly, Lx = len(sites), len(sites[0])
    items = []
    for y in range(Ly):
        for x in range(Lx):
            if (x, y) == tuple(s1):
                t, extra = reduced_impurity(sites[y][x]), ["k1", "b1"]
            elif (x, y) == tuple(s2):
                t, extra = reduced_impurity(sites[y][x]), ["k2", "b2"]
            else:
                t, extra = reduced_tensor(sites[y][x]), []
            ls = [("h", y, x - 1), ("v", y - 1, x), ("h", y, x), ("v", y, x)] + extra
            items.append(_fix_outer(t, ls, y == 0, x == 0, y == Ly - 1, x == Lx - 1))
    t, ls = _contract_sequence(items)
    order = [ls.index(l) for l in ("k1", "k2", "b1", "b2")]
    return t.permute(*order).reshape(d * d, d * d)


def lanczos_ground(Lx, Ly, h, bonds=None, d=2):
    """Lowest eigenvalue of sum_b h_b on the open cluster (scipy eigsh, Lanczos)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    n = Lx * Ly
    bonds = bonds if bonds is not None else cluster_bonds(Lx, Ly)
    idx = [(y1 * Lx + x1, y2 * Lx + x2) for (x1, y1), (x2, y2) in bonds]
    hh = np.asarray(h).reshape(d, d, d, d)

    def mv(v):
        psi = v.reshape([d] * n)
        out = np.zeros_like(psi)
        for i, j in idx:
            t = np.tensordot(hh, psi, axes=([2, 3], [i, j]))
            out += np.moveaxis(t, [0, 1], [i, j])
        return out.reshape(-1)

    op = LinearOperator((d**n, d**n), matvec=mv, dtype=np.float64)
    vals = eigsh(op, k=1, which="SA", tol=1e-12, v0=np.ones(d**n), return_eigenvectors=False)
    return float(vals[0])
