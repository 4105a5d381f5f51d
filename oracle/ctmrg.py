"""Multisite CTMRG with QR+SVD projectors and its reverse mode (oracle, FP64).

Follows Sec. SLF and Fig. 3 of the paper:

* Every site (i, j) of an R x C unit cell owns four corners and four edges
  (Fig. 3(a)).  Leg order of each (this oracle's own convention):
      C_ul[r, d]   T_u[l, d, r]   C_ur[l, d]   T_r[u, l, d]
      C_dr[u, l]   T_d[l, u, r]   C_dl[u, r]   T_l[u, r, d]
  The edge leg toward the centre ("d" of T_u, "l" of T_r, ...) attaches to
  the site's leg on that side.
* A left move processes columns j = 0 .. C-1 in order.  For column j, every
  row i first gets a projector pair (P^(i,j), Q^(i+1,j)) on the cut between
  rows i and i+1, built from the 2x2 cluster of sites (i..i+1, j..j+1) and
  their environments (Fig. 3(c)); then every row updates the left corner,
  edge and corner of site (i, j+1) by absorbing column j (Fig. 3(b)).
  The text (move from T^(i,j) to T^(i,j+1)) is followed where the caption
  says T^(i+1,j).
* Projectors (Eqs. PQ, QRSVD): N = Q_n R_n, S = Q_s R_s, R_n R_s^t = U L V^t,
  P = R_s^t V L~^{-1/2}, Q = R_n^t U L~^{-1/2}, with L~ the chi largest
  singular values.  N is the upper half of the cluster with rows indexed by
  the open right-hand cut and columns by the left cut where P Q^t is
  inserted; S is the lower half, same index order.
* One iteration = left, right, up, down moves (Sec. SLF).  Right, up and down
  moves are left moves of the network rotated by 180, 90 (counterclockwise)
  and 270 degrees.

Readings where the paper is silent:

* Initial environment: a seeded positive random environment supplied as input
  (``from_ring_arrays``).  The trivial boundary (C[0,0] = 1, T[0,0,0] = 1) is
  a fixed point of the nested iteration -- the delta tensors X and Y carry
  index 0 straight through, so every bond density matrix stays rank one --
  and is kept only as ``init_env`` for the tests that show this.
* Pseudo-inverse: L~_k^{-1/2} := 0 when L_k <= CUTOFF * L_1 (CUTOFF = 1e-6).
  Eq. PQ keeps the chi largest singular values; the cutoff removes the ones
  whose singular vectors FP64 cannot resolve.  An SVD in FP64 determines the
  vector of a singular value s_k only to about 1e-16 s_1 / gap_k, and the
  projectors weight it by 1/s_k, so small kept values make the gradient
  depend on the SVD algorithm: the same evaluation with LAPACK's gesvd and
  gesdd drivers gives gradients that differ by up to 4e-4 (relative L2) at a
  cutoff of 1e-8, 1e-6 at 1e-7, 6e-8 at 1e-6 and 2e-9 at 1e-5 (Heisenberg
  D=2, chi=8 and a 2x2-cell Shastry-Sutherland case, 1-20 iterations).  1e-6
  is the smallest cutoff at which the FP64 gradient is reproducible well
  below the 1e-5 parity bar; at D=6, chi=64 it still keeps all 64 values.
* Every updated C and T is divided by its Frobenius norm; the norm is held
  constant under differentiation (the energy does not depend on it).
* Sign gauge of the singular triplets: each right singular vector of rho
  (column of Q_s V) has its entry of largest magnitude (the first one on
  ties) positive, and the left vector follows.  Energies and gradients do
  not depend on it; it makes one CTMRG iteration a map with an element-wise
  fixed point, which the fixed-point gradient (``oracle/fixed_point.py``)
  needs.
* Reverse mode of the projector step: the adjoint of the thin SVD of the
  bond density matrix rho = N S^t = (Q_n U) L (Q_s V)^t over its numerically
  non-zero singular values (s > RANK_TOL * s_1, RANK_TOL = 1e-13; those
  between RANK_TOL and CUTOFF are discarded by the projectors but still
  couple to the kept ones), with the Lorentzian broadening
  F_ij = (s_j^2 - s_i^2) / ((s_j^2 - s_i^2)^2 + EPS * (s_i^2 + s_j^2)^2),
  EPS = 1e-24: it only acts on pairs whose relative gap is at the rounding
  level (numerically degenerate pairs).  A broadening on the absolute scale
  s_1^4 instead damps every coupling among the small kept values (with
  1e-30 s_1^4 the gradient missed finite differences by 2e-2), and a larger
  one (1e-12 is common) biases the gradient visibly.
  P and Q depend on N and S only through this SVD, so this is the exact
  derivative of Eqs. PQ/QRSVD wherever the retained spectrum is
  non-degenerate, and it needs no inverse of R_n or R_s.

Parity: pinned by tests/test_oracle_pins.py (product states, dimer state,
decoupled chains, single vs double layer, finite differences, autograd of
the plain QR+SVD on full-rank inputs).
"""
from __future__ import annotations

import numpy as np
import torch

from .counter import add_qr, add_svd
from .counter import einsum as counted_einsum

DT = torch.float64
CUTOFF = 1e-6
EPS_BROADEN = 1e-24
RANK_TOL = 1e-13
SLOTS = ("C_ul", "T_u", "C_ur", "T_r", "C_dr", "T_d", "C_dl", "T_l")


# ----------------------------------------------------------------------------- projectors
def _qr(A: torch.Tensor):
    """Reduced QR A = Q R by LAPACK (dgeqrf/dorgqr) through scipy.

    torch's CPU QR returned non-finite factors for finite inputs on one of the
    platforms this runs on; scipy's LAPACK build does not.
    """
    import scipy.linalg
    a = A.detach().numpy()
    if not np.isfinite(a).all():
        raise FloatingPointError("non-finite input to QR")
    Q, R = scipy.linalg.qr(a, mode="economic")
    add_qr(*a.shape)
    return torch.from_numpy(Q), torch.from_numpy(R)


def _svd(M: torch.Tensor):
    """Full SVD M = U diag(s) V^t by LAPACK's QR-iteration driver (dgesvd).

    The divide-and-conquer driver (dgesdd) aborted on some of these badly
    scaled bond matrices on one of the platforms this runs on; dgesvd does not.
    """
    import scipy.linalg
    m = M.detach().numpy()
    if not np.isfinite(m).all():
        raise FloatingPointError("non-finite input to SVD")
    U, s, Vh = scipy.linalg.svd(m, full_matrices=True, lapack_driver="gesvd")
    add_svd(*m.shape)
    return torch.from_numpy(U), torch.from_numpy(s), torch.from_numpy(Vh.T.copy())


def _sign_gauge(U: torch.Tensor, V: torch.Tensor, Qs: torch.Tensor):
    """Flip (u_k, v_k) together so that the largest-magnitude entry of Q_s v_k is positive."""
    Vp = Qs @ V
    idx = Vp.abs().argmax(dim=0)
    sg = torch.sign(Vp[idx, torch.arange(Vp.shape[1])])
    sg = torch.where(sg == 0, torch.ones_like(sg), sg)
    return U * sg, V * sg


def _broadened_inverse_gaps(s: torch.Tensor, nz: torch.Tensor) -> torch.Tensor:
    """F_ij = (s_j^2 - s_i^2)/((s_j^2 - s_i^2)^2 + EPS (s_i^2 + s_j^2)^2) on the non-zero set, 0 elsewhere."""
    s2 = s * s
    diff = s2[None, :] - s2[:, None]
    scale = s2[None, :] + s2[:, None]
    F = diff / (diff * diff + EPS_BROADEN * scale * scale)
    mask = nz[:, None] & nz[None, :]
    F = torch.where(mask, F, torch.zeros_like(F))
    F.fill_diagonal_(0.0)
    return F


class Projectors(torch.autograd.Function):
    """(N, S) -> (P, Q) of Eqs. PQ/QRSVD, with the adjoint described in the module docstring."""

    @staticmethod
    def forward(ctx, N: torch.Tensor, S: torch.Tensor, chi: int):
        Qn, Rn = _qr(N)
        Qs, Rs = _qr(S)
        M = Rn @ Rs.T
        U, s, V = _svd(M)
        U, V = _sign_gauge(U, V, Qs)
        k = s.shape[0]
        kept = min(chi, k)
        cut = CUTOFF * s[0]
        lam = s[:kept]
        inv = torch.where(lam > cut, lam.clamp_min(1e-300).rsqrt(), torch.zeros_like(lam))
        n_l = N.shape[1]
        P = torch.zeros(n_l, chi, dtype=DT)
        Q = torch.zeros(n_l, chi, dtype=DT)
        P[:, :kept] = (Rs.T @ V[:, :kept]) * inv
        Q[:, :kept] = (Rn.T @ U[:, :kept]) * inv
        nz = s > RANK_TOL * s[0]
        Up = (Qn @ U) * nz
        Vp = (Qs @ V) * nz
        ctx.save_for_backward(N, S, Up, Vp, s, inv)
        ctx.kept = kept
        return P, Q

    @staticmethod
    def backward(ctx, dP, dQ):
        N, S, Up, Vp, s, inv = ctx.saved_tensors
        kept = ctx.kept
        k = s.shape[0]
        dP, dQ = dP[:, :kept], dQ[:, :kept]
        W = Vp[:, :kept] * inv
        Z = Up[:, :kept] * inv
        dS = W @ dP.T
        dW = S @ dP
        dN = Z @ dQ.T
        dZ = N @ dQ
        n_r = N.shape[0]
        dU = torch.zeros(n_r, k, dtype=DT)
        dV = torch.zeros(n_r, k, dtype=DT)
        dU[:, :kept] = dZ * inv
        dV[:, :kept] = dW * inv
        dl = torch.zeros(k, dtype=DT)
        dl[:kept] = -0.5 * inv**3 * ((dZ * Up[:, :kept]).sum(0) + (dW * Vp[:, :kept]).sum(0))
        nz = s > RANK_TOL * s[0]
        F = _broadened_inverse_gaps(s, nz)
        A = Up.T @ dU
        B = Vp.T @ dV
        J = F * (A - A.T)
        K = F * (B - B.T)
        core = J * s[None, :] + s[:, None] * K + torch.diag(dl)
        sinv = torch.where(nz, 1.0 / s.clamp_min(1e-300), torch.zeros_like(s))
        Eu = (dU - Up @ A) * sinv[None, :]
        Ev = (dV - Vp @ B) * sinv[None, :]
        drho = Up @ core @ Vp.T + Eu @ Vp.T + Up @ Ev.T
        dN = dN + drho @ S
        dS = dS + drho.T @ N
        return dN, dS, None


def projectors(N, S, chi):
    return Projectors.apply(N, S, chi)


def projectors_plain(N, S, chi):
    """Same function through torch's own QR/SVD autograd (valid for full-rank, non-degenerate inputs)."""
    Qn, Rn = torch.linalg.qr(N, mode="reduced")
    Qs, Rs = torch.linalg.qr(S, mode="reduced")
    U, s, Vh = torch.linalg.svd(Rn @ Rs.T)
    inv = s[:chi].rsqrt()
    return (Rs.T @ Vh.T[:, :chi]) * inv, (Rn.T @ U[:, :chi]) * inv


# ----------------------------------------------------------------------------- environment
def init_env(grid, chi: int) -> dict:
    """Trivial boundary: C[0,0]=1, T[0,0,0]=1, zero-padded to chi."""
    R, C = len(grid), len(grid[0])
    env = {k: [[None] * C for _ in range(R)] for k in SLOTS}
    for i in range(R):
        for j in range(C):
            bl, bu, br, bd = grid[i][j].shape[:4]
            for k in ("C_ul", "C_ur", "C_dr", "C_dl"):
                c = torch.zeros(chi, chi, dtype=DT)
                c[0, 0] = 1.0
                env[k][i][j] = c
            for k, b in (("T_u", bu), ("T_r", br), ("T_d", bd), ("T_l", bl)):
                t = torch.zeros(chi, b, chi, dtype=DT)
                t[0, 0, 0] = 1.0
                env[k][i][j] = t
    return env


def from_ring_arrays(arrays, R: int, C: int) -> dict:
    """Environment from per-site arrays in the ring convention used for inputs.

    ``arrays[i*C + j]`` lists the 8 tensors of site (i, j) in SLOTS order with
    legs (prev, [in,] next) clockwise around the site:
    C_ul [down, right], T_u [left, in, right], C_ur [left, down],
    T_r [up, in, down], C_dr [up, left], T_d [right, in, left],
    C_dl [right, up], T_l [down, in, up].
    """
    conv = {"C_ul": (1, 0), "T_u": (0, 1, 2), "C_ur": (0, 1), "T_r": (0, 1, 2),
            "C_dr": (0, 1), "T_d": (2, 1, 0), "C_dl": (1, 0), "T_l": (2, 1, 0)}
    env = {k: [[None] * C for _ in range(R)] for k in SLOTS}
    for i in range(R):
        for j in range(C):
            for k, a in zip(SLOTS, arrays[i * C + j]):
                env[k][i][j] = torch.as_tensor(a, dtype=DT).permute(*conv[k]).contiguous()
    return env


def to_ring_arrays(env) -> list:
    """Inverse of ``from_ring_arrays`` (numpy arrays)."""
    conv = {"C_ul": (1, 0), "T_u": (0, 1, 2), "C_ur": (0, 1), "T_r": (0, 1, 2),
            "C_dr": (0, 1), "T_d": (2, 1, 0), "C_dl": (1, 0), "T_l": (2, 1, 0)}
    R, C = len(env["C_ul"]), len(env["C_ul"][0])
    return [[env[k][i][j].detach().permute(*conv[k]).contiguous().numpy() for k in SLOTS]
            for i in range(R) for j in range(C)]


def rotate_ccw(grid, env):
    """Rotate network and environment counterclockwise by 90 degrees.

    Site (i, j) of an R x C cell moves to (C-1-j, i) of a C x R cell; a site's
    up leg becomes its left leg, right -> up, down -> right, left -> down.
    """
    R, C = len(grid), len(grid[0])
    ng = [[None] * R for _ in range(C)]
    ne = {k: [[None] * R for _ in range(C)] for k in SLOTS}
    for i in range(R):
        for j in range(C):
            ii, jj = C - 1 - j, i
            ng[ii][jj] = grid[i][j].permute(1, 2, 3, 0)
            if env is None:
                continue
            ne["C_ul"][ii][jj] = env["C_ur"][i][j].permute(1, 0)
            ne["T_u"][ii][jj] = env["T_r"][i][j]
            ne["C_ur"][ii][jj] = env["C_dr"][i][j]
            ne["T_r"][ii][jj] = env["T_d"][i][j].permute(2, 1, 0)
            ne["C_dr"][ii][jj] = env["C_dl"][i][j].permute(1, 0)
            ne["T_d"][ii][jj] = env["T_l"][i][j]
            ne["C_dl"][ii][jj] = env["C_ul"][i][j]
            ne["T_l"][ii][jj] = env["T_u"][i][j].permute(2, 1, 0)
    return ng, (ne if env is not None else None)


def rotate(grid, env, q: int):
    for _ in range(q % 4):
        grid, env = rotate_ccw(grid, env)
    return grid, env


# ----------------------------------------------------------------------------- half systems
def _corner_ul(C, Tu, Tl, a):
    x1 = counted_einsum("xy,xpz->ypz", C, Tu)
    x2 = counted_einsum("ypz,yqw->pzqw", x1, Tl)
    return counted_einsum("pzqw,qpst->wtzs", x2, a)          # [T_l.d, a.d | T_u.r, a.r]


def _corner_ur(Tu, C, Tr, a):
    x1 = counted_einsum("zpx,xy->zpy", Tu, C)
    x2 = counted_einsum("zpy,yqv->zpqv", x1, Tr)
    return counted_einsum("zpqv,spqt->zstv", x2, a)          # [T_u.l, a.l | a.d, T_r.d]


def _corner_dl(Tl, C, Td, a):
    x1 = counted_einsum("wqy,yx->wqx", Tl, C)
    x2 = counted_einsum("wqx,xpz->wqpz", x1, Td)
    return counted_einsum("wqpz,qtsp->wtzs", x2, a)          # [T_l.u, a.u | T_d.r, a.r]


def _corner_dr(Tr, C, Td, a):
    x1 = counted_einsum("vqy,yx->vqx", Tr, C)
    x2 = counted_einsum("vqx,zpx->vqzp", x1, Td)
    return counted_einsum("vqzp,stqp->zstv", x2, a)          # [T_d.l, a.l | a.u, T_r.u]


def _half(G_left, G_right):
    """[w, t | z, s] x [z, s | T, v] -> matrix [(T, v), (w, t)]."""
    X = counted_einsum("wtzs,zsTv->Tvwt", G_left, G_right)
    return X.reshape(X.shape[0] * X.shape[1], X.shape[2] * X.shape[3])


def cluster_halves(grid, env, i, j):
    """N (upper) and S (lower) for the cut between rows i, i+1 at columns j, j+1."""
    R, C = len(grid), len(grid[0])
    ip, jp = (i + 1) % R, (j + 1) % C
    e = env
    Gul = _corner_ul(e["C_ul"][i][j], e["T_u"][i][j], e["T_l"][i][j], grid[i][j])
    Gur = _corner_ur(e["T_u"][i][jp], e["C_ur"][i][jp], e["T_r"][i][jp], grid[i][jp])
    Gdl = _corner_dl(e["T_l"][ip][j], e["C_dl"][ip][j], e["T_d"][ip][j], grid[ip][j])
    Gdr = _corner_dr(e["T_r"][ip][jp], e["C_dr"][ip][jp], e["T_d"][ip][jp], grid[ip][jp])
    return _half(Gul, Gur), _half(Gdl, Gdr)


# ----------------------------------------------------------------------------- moves
def _normalize(t):
    return t / t.norm().detach()


def left_move(grid, env, chi, spectra=None):
    """One left move (all columns in order) on an R x C cell; returns the new env dict."""
    R, C = len(grid), len(grid[0])
    env = {k: [row[:] for row in env[k]] for k in SLOTS}
    for j in range(C):
        jp = (j + 1) % C
        Ps, Qs = [None] * R, [None] * R
        for i in range(R):
            N, S = cluster_halves(grid, env, i, j)
            P, Q = projectors(N, S, chi)
            bP = grid[i][j].shape[3]                 # a[i,j].d
            bQ = grid[(i + 1) % R][j].shape[1]        # a[i+1,j].u
            Ps[i] = P.reshape(chi, bP, chi)
            Qs[i] = Q.reshape(chi, bQ, chi)
            if spectra is not None:
                spectra.append(_spectrum(N.detach(), S.detach(), chi))
        new = []
        for i in range(R):
            im = (i - 1) % R
            Cul = counted_einsum("xy,xpr,ypk->rk", env["C_ul"][i][j], env["T_u"][i][j], Ps[im])
            x1 = counted_einsum("yqz,qpsw->yzpsw", env["T_l"][i][j], grid[i][j])
            x2 = counted_einsum("yzpsw,ypu->zswu", x1, Qs[im])
            Tl = counted_einsum("zswu,zwd->usd", x2, Ps[i])
            Cdl = counted_einsum("yx,xpr,ypu->ur", env["C_dl"][i][j], env["T_d"][i][j], Qs[i])
            new.append((_normalize(Cul), _normalize(Tl), _normalize(Cdl)))
        for i in range(R):
            env["C_ul"][i][jp], env["T_l"][i][jp], env["C_dl"][i][jp] = new[i]
    return env


def _spectrum(N, S, chi):
    with torch.no_grad():
        _, Rn = _qr(N)
        _, Rs = _qr(S)
        s = _svd(Rn @ Rs.T)[1][:chi]
        return s / s.sum()


def move(grid, env, chi, direction: str, spectra=None):
    q = {"left": 0, "up": 1, "right": 2, "down": 3}[direction]
    g, e = rotate(grid, env, q)
    e = left_move(g, e, chi, spectra)
    _, e = rotate(g, e, 4 - q)
    return e


def ctmrg(grid, chi: int, n_iter: int, env=None, spectra_log=None):
    """n_iter iterations of (left, right, up, down) from the trivial boundary (or ``env``).

    ``spectra_log``, if a list, receives per iteration the list of normalised
    truncated spectra s~/sum(s~) of every projector pair, in execution order.
    """
    if env is None:
        env = init_env(grid, chi)
    for _ in range(n_iter):
        spectra = [] if spectra_log is not None else None
        for direction in ("left", "right", "up", "down"):
            env = move(grid, env, chi, direction, spectra)
        if spectra_log is not None:
            spectra_log.append(spectra)
    return env


def spectrum_change(prev, cur) -> float:
    """delta = max over projector pairs of || s~/|s~|_1 - s~_prev/|s~_prev|_1 ||_inf."""
    return max(float((a - b).abs().max()) for a, b in zip(prev, cur))
