"""Python binding of libctm: the same calls as include/ctm.h on torch device memory.

Every step of the path runs inside libctm's CUDA kernels; this module only
marshals arguments (device pointers of torch tensors, the current stream).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


class CTMError(RuntimeError):
    def __init__(self, status, where):
        lib = _lib.load()
        super().__init__(f"{where}: {lib.ctm_error_string(status).decode()} (status {status})")
        self.status = status


def _check(status, where):
    if status != 0:
        raise CTMError(status, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class CTM:
    """One problem size: PEPS cell Lx x Ly, d, D, chi, precision, Hamiltonian terms.

    ``terms``: iterable of (x, y, kind, coupling, h) with h a d^2 x d^2 array.
    """

    def __init__(self, Lx, Ly, d, D, chi, terms, precision="fp64", cutoff=1e-6, adjoint_eps=1e-24):
        self.lib = _lib.load()
        self.Lx, self.Ly, self.d, self.D, self.chi = Lx, Ly, d, D, chi
        self.precision = precision
        self.cutoff = cutoff
        self._h = [np.ascontiguousarray(np.asarray(t[4], dtype=np.float64)) for t in terms]
        arr = (_lib.CtmTerm * len(self._h))()
        for k, t in enumerate(terms):
            arr[k].x, arr[k].y, arr[k].kind, arr[k].coupling = int(t[0]), int(t[1]), int(t[2]), float(t[3])
            arr[k].h = self._h[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        desc = _lib.CtmDesc(Lx, Ly, d, D, chi, _lib.PRECISIONS[precision], len(self._h), arr, cutoff, adjoint_eps, 0)
        self._terms = arr
        h = ctypes.c_void_p()
        _check(self.lib.ctm_create(ctypes.byref(desc), ctypes.byref(h)), "ctm_create")
        self.handle = h
        self.n_terms = len(self._h)

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.ctm_destroy(self.handle)
            self.handle = None

    @property
    def env_numel(self):
        return int(self.lib.ctm_env_numel(self.handle))

    @property
    def kernel_launches(self):
        return int(self.lib.ctm_kernel_launches(self.handle))

    def init(self, A, env0=None):
        """A: cuda float64 [Lx*Ly, d, D, D, D, D]; env0: cuda float64 flat ring-layout environment."""
        assert A.is_cuda and A.dtype == torch.float64 and A.is_contiguous()
        if env0 is not None:
            assert env0.is_cuda and env0.dtype == torch.float64 and env0.numel() == self.env_numel
        _check(self.lib.ctm_init(self.handle, _ptr(A), _ptr(env0), _stream()), "ctm_init")

    def step(self, n_iter):
        delta = ctypes.c_double(-1.0)
        _check(self.lib.ctm_step(self.handle, int(n_iter), ctypes.byref(delta), _stream()), "ctm_step")
        return delta.value

    def energy(self, per_bond=False):
        e = torch.empty(1, dtype=torch.float64, device="cuda")
        eb = torch.empty(self.n_terms, dtype=torch.float64, device="cuda") if per_bond else None
        _check(self.lib.ctm_energy(self.handle, _ptr(e), _ptr(eb), _stream()), "ctm_energy")
        return (e, eb) if per_bond else e

    def magnetization(self):
        """Eq. Mag1: (per-site (<Sx>, <Sy>, <Sz>) as a cuda [Lx*Ly, 3] tensor, M as a cuda [1] tensor)."""
        m = torch.empty(self.Lx * self.Ly, 3, dtype=torch.float64, device="cuda")
        M = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(self.lib.ctm_magnetization(self.handle, _ptr(m), _ptr(M), _stream()), "ctm_magnetization")
        return m, M

    def plaquette_order(self, terms_a, terms_b):
        """Eq. Mag2 from the bond values of two lists of term indices: a cuda [1] tensor."""
        a = (ctypes.c_int * len(terms_a))(*terms_a)
        b = (ctypes.c_int * len(terms_b))(*terms_b)
        Mp = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(self.lib.ctm_plaquette_order(self.handle, a, len(terms_a), b, len(terms_b), _ptr(Mp), _stream()),
               "ctm_plaquette_order")
        return Mp

    def grad(self, n_iter, dA=None, e=None):
        nA = self.Lx * self.Ly * self.d * self.D ** 4
        dA = dA if dA is not None else torch.empty(self.Lx * self.Ly, self.d, self.D, self.D, self.D, self.D,
                                                  dtype=torch.float64, device="cuda")
        e = e if e is not None else torch.empty(1, dtype=torch.float64, device="cuda")
        assert dA.numel() == nA
        _check(self.lib.ctm_grad(self.handle, int(n_iter), _ptr(e), _ptr(dA), _stream()), "ctm_grad")
        return e, dA

    def grad_fixed_point(self, max_terms=200, tol=1e-10, dA=None, e=None):
        """Fixed-point gradient at the current (converged) environment: (e, dA, terms, residual)."""
        nA = self.Lx * self.Ly * self.d * self.D ** 4
        dA = dA if dA is not None else torch.empty(self.Lx * self.Ly, self.d, self.D, self.D, self.D, self.D,
                                                  dtype=torch.float64, device="cuda")
        e = e if e is not None else torch.empty(1, dtype=torch.float64, device="cuda")
        assert dA.numel() == nA
        info = (ctypes.c_double * 2)()
        _check(self.lib.ctm_grad_fixed_point(self.handle, int(max_terms), float(tol), _ptr(e), _ptr(dA), info,
                                             _stream()), "ctm_grad_fixed_point")
        return e, dA, int(info[0]), float(info[1])

    def set_limits(self, max_sweeps=0, spin_limit=0):
        """Sweep limit of the Jacobi SVD and spin limit of the bounded device waits (0: default)."""
        _check(self.lib.ctm_set_limits(self.handle, int(max_sweeps), int(spin_limit)), "ctm_set_limits")

    def profile(self, enable=True):
        _check(self.lib.ctm_profile(self.handle, int(bool(enable))), "ctm_profile")

    def profile_read(self):
        """{class: (ms, launches, flops, bytes)} for every kernel class since profile(True)."""
        out = {}
        for name, c in _lib.PROF_CLASSES.items():
            ms, n, fl, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            _check(self.lib.ctm_profile_read(self.handle, c, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                             ctypes.byref(by)), "ctm_profile_read")
            out[name] = (ms.value, n.value, fl.value, by.value)
        return out

    def spectra(self, iteration, max_pairs=256, max_vals=None):
        """Singular values of every projector pair of one iteration: (n_pairs, max_vals) numpy array."""
        max_vals = max_vals or self.chi
        out = np.zeros((max_pairs, max_vals), dtype=np.float64)
        n = ctypes.c_int(0)
        _check(self.lib.ctm_get_spectra(self.handle, int(iteration), out.ctypes.data_as(ctypes.c_void_p), max_pairs,
                                        max_vals, ctypes.byref(n)), "ctm_get_spectra")
        return out[: n.value]

    def get_env(self):
        out = torch.empty(self.env_numel, dtype=torch.float64, device="cuda")
        _check(self.lib.ctm_get_env(self.handle, _ptr(out), _stream()), "ctm_get_env")
        return out

    def set_env(self, env):
        assert env.is_cuda and env.dtype == torch.float64 and env.numel() == self.env_numel
        _check(self.lib.ctm_set_env(self.handle, _ptr(env), _stream()), "ctm_set_env")


def svd(M):
    """Batched FP64 SVD of square matrices (cuda float64 [batch, r, r]) by libctm's Jacobi kernels.

    Returns U, s, V with M[b] = U[b] diag(s[b]) V[b]^t, s descending."""
    lib = _lib.load()
    assert M.is_cuda and M.dtype == torch.float64 and M.dim() == 3 and M.shape[1] == M.shape[2]
    M = M.contiguous()
    b, r = M.shape[0], M.shape[1]
    U = torch.empty_like(M)
    V = torch.empty_like(M)
    s = torch.empty(b, r, dtype=torch.float64, device=M.device)
    _check(lib.ctm_svd(_ptr(M), b, r, _ptr(U), _ptr(s), _ptr(V), _stream()), "ctm_svd")
    return U, s, V


class CTMEnergy(torch.autograd.Function):
    """E(A) after n_iter CTMRG iterations from env0; backward returns dE/dA from ctm_grad."""

    @staticmethod
    def forward(ctx, A, ctm, env0, n_iter):
        ctm.init(A.detach().contiguous(), env0)
        e, dA = ctm.grad(n_iter)
        ctx.save_for_backward(dA)
        return e[0].clone()

    @staticmethod
    def backward(ctx, g):
        (dA,) = ctx.saved_tensors
        return g * dA, None, None, None
