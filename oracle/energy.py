"""Impurity reduced density matrices and the energy estimator (oracle, FP64).

Eq. ExpH: E = <Psi|H|Psi> / <Psi|Psi>.  Each bond term is evaluated with its
own reduced density matrix: the block of the network that holds both sites,
closed by the environment (Fig. 3(a)), with the physical line of each of the
two sites cut open (the impurity tensors of Sec. NTN).  Reading: per bond
e_b = Tr(rho_b h_b) / Tr(rho_b), and E per site = sum_b J_b e_b / (Lx Ly).

Nested blocks (rows x cols of nested sites, upper-left at (2y, 2x)):
  H bond (x,y)-(x+1,y):            2 x 4, open Y at (0,1) and (0,3)
  V bond (x,y)-(x,y+1):            4 x 2, open Y at (0,1) and (2,1)
  DIAG_DR (x,y)-(x+1,y+1):         4 x 4, open Y at (0,1) and (2,3)
  DIAG_UR (x+1,y)-(x,y+1):         4 x 4, open Y at (0,3) and (2,1)
Double-layer blocks use the reduced tensors with the open impurity tensor.

rho is returned as a d^2 x d^2 matrix, rows (ket s1, ket s2), columns
(bra s1, bra s2).

Parity: pinned by the exact finite-cluster tests and the closed-form product
and dimer states.
"""
from __future__ import annotations

import itertools
import math

import torch

from .counter import einsum as counted_einsum

from .nested import (DT, double_cell, nested_cell, reduced_impurity, y_impurity)

H_, V_, DR_, UR_ = 0, 1, 2, 3


# ----------------------------------------------------------------------------- label contraction
def contract_pair(a, b):
    ta, la = a
    tb, lb = b
    shared = [l for l in la if l in lb]
    out = [l for l in la if l not in shared] + [l for l in lb if l not in shared]
    m = {l: k for k, l in enumerate(dict.fromkeys(list(la) + list(lb)))}
    t = counted_einsum(ta, [m[l] for l in la], tb, [m[l] for l in lb], [m[l] for l in out])
    return t, out


def _dims(items):
    dims = {}
    for t, ls in items:
        for l, n in zip(ls, t.shape):
            dims[l] = n
    return dims


def contract_greedy(items):
    """Contract a list of (tensor, labels) pairwise, always taking the connected pair
    with the smallest result (ties: fewest multiply-adds)."""
    items = list(items)
    dims = _dims(items)
    while len(items) > 1:
        best = None
        for p in range(len(items)):
            for q in range(p + 1, len(items)):
                lp, lq = items[p][1], items[q][1]
                shared = set(lp) & set(lq)
                if not shared:
                    continue
                out = (set(lp) | set(lq)) - shared
                size = math.prod(dims[l] for l in out)
                cost = size * math.prod(dims[l] for l in shared)
                key = (size, cost)
                if best is None or key < best[0]:
                    best = (key, p, q)
        if best is None:   # disconnected: outer product of the first two
            best = (None, 0, 1)
        _, p, q = best
        new = contract_pair(items[p], items[q])
        items = [it for k, it in enumerate(items) if k not in (p, q)] + [new]
    return items[0]


# ----------------------------------------------------------------------------- block networks
def block_rdm(grid, env, i0, j0, h, w, imps):
    """Contract an h x w block at (i0, j0) with its environment.

    ``imps`` maps block positions (a, b) to ``(tensor, ket_label, bra_label)``:
    a site tensor with two trailing open legs.  Returns (tensor, open labels).
    """
    R, C = len(grid), len(grid[0])
    lab = itertools.count()
    Hb = {(a, b): next(lab) for a in range(h) for b in range(-1, w)}
    Vb = {(a, b): next(lab) for a in range(-1, h) for b in range(w)}
    TU = [next(lab) for _ in range(w + 1)]
    TD = [next(lab) for _ in range(w + 1)]
    TL = [next(lab) for _ in range(h + 1)]
    TR = [next(lab) for _ in range(h + 1)]
    groups = {}

    def grp(a, b):
        return (a // 2, b // 2)

    def add(g, t, ls):
        groups.setdefault(g, []).append((t, ls))

    for a in range(h):
        for b in range(w):
            ls = [Hb[a, b - 1], Vb[a - 1, b], Hb[a, b], Vb[a, b]]
            if (a, b) in imps:
                t, ka, kb = imps[(a, b)]
                add(grp(a, b), t, ls + [ka, kb])
            else:
                add(grp(a, b), grid[(i0 + a) % R][(j0 + b) % C], ls)
    I = lambda a: (i0 + a) % R
    J = lambda b: (j0 + b) % C
    add(grp(0, 0), env["C_ul"][I(0)][J(0)], [TU[0], TL[0]])
    add(grp(0, w - 1), env["C_ur"][I(0)][J(w - 1)], [TU[w], TR[0]])
    add(grp(h - 1, w - 1), env["C_dr"][I(h - 1)][J(w - 1)], [TR[h], TD[w]])
    add(grp(h - 1, 0), env["C_dl"][I(h - 1)][J(0)], [TL[h], TD[0]])
    for b in range(w):
        add(grp(0, b), env["T_u"][I(0)][J(b)], [TU[b], Vb[-1, b], TU[b + 1]])
        add(grp(h - 1, b), env["T_d"][I(h - 1)][J(b)], [TD[b], Vb[h - 1, b], TD[b + 1]])
    for a in range(h):
        add(grp(a, 0), env["T_l"][I(a)][J(0)], [TL[a], Hb[a, -1], TL[a + 1]])
        add(grp(a, w - 1), env["T_r"][I(a)][J(w - 1)], [TR[a], Hb[a, w - 1], TR[a + 1]])
    parts = [contract_greedy(groups[g]) for g in sorted(groups)]
    return contract_greedy(parts)


def _rho_matrix(t, labels, k1, k2, b1, b2, d):
    order = [labels.index(l) for l in (k1, k2, b1, b2)]
    return t.permute(*order).reshape(d * d, d * d)


def bond_energy(rho, h):
    """Tr(rho h) / Tr(rho) for a d^2 x d^2 density matrix (rows ket, columns bra)."""
    return counted_einsum("ab,ba->", rho, h) / torch.trace(rho)


_NESTED_BLOCK = {H_: (2, 4, (0, 1), (0, 3)), V_: (4, 2, (0, 1), (2, 1)),
                 DR_: (4, 4, (0, 1), (2, 3)), UR_: (4, 4, (0, 3), (2, 1))}
_DOUBLE_BLOCK = {H_: (1, 2, (0, 0), (0, 1)), V_: (2, 1, (0, 0), (1, 0)),
                 DR_: (2, 2, (0, 0), (1, 1)), UR_: (2, 2, (0, 1), (1, 0))}


def nested_rdm(As, Lx, Ly, grid, env, x, y, kind):
    d, D = As[0].shape[0], As[0].shape[1]
    Yi = y_impurity(D, d)
    h, w, s1, s2 = _NESTED_BLOCK[kind]
    imps = {s1: (Yi, "k1", "b1"), s2: (Yi, "k2", "b2")}
    t, ls = block_rdm(grid, env, 2 * y, 2 * x, h, w, imps)
    return _rho_matrix(t, ls, "k1", "k2", "b1", "b2", d)


def double_rdm(As, Lx, Ly, grid, env, x, y, kind):
    d = As[0].shape[0]
    h, w, s1, s2 = _DOUBLE_BLOCK[kind]
    imps = {}
    for (a, b), (k, bb) in ((s1, ("k1", "b1")), (s2, ("k2", "b2"))):
        p = ((y + a) % Ly) * Lx + (x + b) % Lx
        imps[(a, b)] = (reduced_impurity(As[p]), k, bb)
    t, ls = block_rdm(grid, env, y, x, h, w, imps)
    return _rho_matrix(t, ls, "k1", "k2", "b1", "b2", d)


def energy(As, Lx, Ly, env, terms, layer="nested", grid=None, per_bond=None):
    """Energy per PEPS site from a converged (or fixed-iteration) environment."""
    if grid is None:
        grid = nested_cell(As, Lx, Ly) if layer == "nested" else double_cell(As, Lx, Ly)
    rdm = nested_rdm if layer == "nested" else double_rdm
    total = torch.zeros((), dtype=DT)
    for t in terms:
        h = torch.as_tensor(t.h, dtype=DT)
        e = bond_energy(rdm(As, Lx, Ly, grid, env, t.x, t.y, t.kind), h)
        if per_bond is not None:
            per_bond.append(float(e.detach()))
        total = total + t.coupling * e
    return total / (Lx * Ly)
