"""Multiply-add counter of the oracle (test infrastructure, like the rest of this package).

Every pairwise contraction of the oracle goes through ``einsum`` below, which adds the product
of the sizes of all distinct labels of the two operands (the multiply-adds of the contraction
written as loops) to ``MACS["contraction"]``; the QR and SVD helpers add the standard Householder
and Golub-Kahan counts.  Only the forward pass is counted (the reverse mode runs inside torch's
autograd); counting is always on and costs a dictionary update per call.
"""
from __future__ import annotations

import torch

MACS = {"contraction": 0, "qr": 0, "svd": 0}


def reset():
    for k in MACS:
        MACS[k] = 0


def _macs_sublist(args):
    dims = {}
    ops = args[:-1] if len(args) % 2 == 1 else args
    for t, labels in zip(ops[0::2], ops[1::2]):
        for l, n in zip(labels, t.shape):
            dims[l] = int(n)
    m = 1
    for n in dims.values():
        m *= n
    return m


def _macs_string(eq, ops):
    lhs = eq.replace(" ", "").split("->")[0]
    dims = {}
    for term, t in zip(lhs.split(","), ops):
        for c, n in zip(term, t.shape):
            dims[c] = int(n)
    m = 1
    for n in dims.values():
        m *= n
    return m


def einsum(*args):
    """torch.einsum with the multiply-adds of the call added to MACS["contraction"]."""
    if isinstance(args[0], str):
        MACS["contraction"] += _macs_string(args[0], args[1:]) if len(args) > 2 else 0
    else:
        MACS["contraction"] += _macs_sublist(args) if len(args) >= 4 else 0
    return torch.einsum(*args)


def add_qr(m: int, n: int):
    """Householder QR of an m x n matrix (m >= n): 2 m n^2 - 2 n^3 / 3 flops, half as multiply-adds."""
    k = min(m, n)
    MACS["qr"] += int((2 * m * n * k - 2 * k ** 3 / 3) / 2)


def add_svd(m: int, n: int):
    """SVD of an m x n matrix with both factors (Golub-Kahan bidiagonalisation + QR iteration):
    about 4 m n^2 + 8 n^3 flops for m >= n (Golub & Van Loan, Sec. 8.6), half as multiply-adds."""
    a, b = max(m, n), min(m, n)
    MACS["svd"] += int((4 * a * b * b + 8 * b ** 3) / 2)
