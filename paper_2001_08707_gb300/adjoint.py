"""Differentiable Green's-function spectrum: a torch.autograd.Function with a
hand-written adjoint.

For H(theta) = sum_t theta_t H_t (real symmetric terms) and shifts z_k,

    A_k(theta) = -(1/pi) Im b^T G(z_k) b,   G(z) = (z I - H)^{-1}   (Eq. 2).

dG/dtheta_t = G H_t G and G^T = G give dA_k/dtheta_t = -(1/pi) Im(x_k^T H_t x_k)
with x_k = G(z_k) b (Eq. 4-5), so the backward pass needs only the forward
solution vectors: no second solve when the left and right vectors are the same.
The forward pass is one full-mode kw_solve; the backward pass is kw_bilinear
over the saved x_k.  For a left vector a different from b (GreenBilinear),
G_ab(z_k) = a^T G(z_k) b has dG_ab/dtheta_t = y_k^T H_t x_k with y_k = G(z_k) a
from a second full-mode solve on the same shifts.  With FP32 shift storage
(kw_set_shift_storage) the saved vectors are complex FP32 and the backward pass
is kw_bilinear_c64; the forward values come from the projected recurrences in
the seed form's precision either way.  This module only assembles the inputs
and the final K x nterm contraction.
"""
from __future__ import annotations

import numpy as np

from paper_2001_08707_gb300 import komega as kw


class TermSet:
    """The parameter matrices on their merged sparsity pattern.

    values(theta) gives the values of H(theta) on the merged pattern with one
    scatter-add per term; device copies of every term feed kw_bilinear."""

    def __init__(self, terms):
        m = terms[0].m
        rows = [np.repeat(np.arange(m, dtype=np.int64), np.diff(t.rowptr)) for t in terms]
        keys = [r * m + t.col.astype(np.int64) for r, t in zip(rows, terms)]
        allk = np.unique(np.concatenate(keys))
        self.m = m
        self.col = (allk % m).astype(np.int32)
        counts = np.bincount(allk // m, minlength=m)
        self.rowptr = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(counts, out=self.rowptr[1:])
        self.index = [np.searchsorted(allk, k) for k in keys]
        self.vals = [t.val.astype(np.float64) for t in terms]
        self._terms = terms
        self._dev = None

    @property
    def device_terms(self):
        """(rowptr, col, val) CUDA tensors of every term, for kw_bilinear."""
        if self._dev is None:
            import torch

            self._dev = [(torch.as_tensor(t.rowptr, device="cuda"), torch.as_tensor(t.col, device="cuda"),
                          torch.as_tensor(t.val, device="cuda")) for t in self._terms]
        return self._dev

    def values(self, theta) -> np.ndarray:
        v = np.zeros(self.col.size, dtype=np.float64)
        for th, idx, val in zip(np.asarray(theta, dtype=np.float64), self.index, self.vals):
            v[idx] += th * val          # indices within one term are distinct
        return v


class GreenSpectrum:
    """A(theta) = -(1/pi) Im b^T G(z_k) b for all shifts, differentiable in theta."""

    def __init__(self, terms, b, z, prec: str = "df64", tol: float = 1e-10, maxiter: int = 200000,
                 shift_fp32: bool = False):
        import torch

        self.terms = TermSet(terms)
        self.b = torch.as_tensor(np.asarray(b, dtype=np.float64), device="cuda")
        self.z = np.asarray(z, dtype=np.complex128)
        self.solver = kw.Solver(prec, tol=tol, maxiter=maxiter)
        self.solver.set_shift_storage(shift_fp32)
        self.rowptr = torch.as_tensor(self.terms.rowptr, device="cuda")
        self.col = torch.as_tensor(self.terms.col, device="cuda")
        self.last = None

    def solve(self, theta):
        """Forward solve for the given parameters; returns (A [K] numpy, x [K, m] device)."""
        import torch

        vals = torch.as_tensor(self.terms.values(theta), device="cuda")
        self.solver.set_csr(self.rowptr, self.col, vals)
        r = self.solver.solve(self.b, self.z, full=True)
        if r.status != "KW_OK":
            raise kw.KomegaError(kw.KW_NOT_CONVERGED, f"forward solve: {r.status} after {r.iters} iterations")
        self.last = r
        return -np.imag(r.proj[:, 0]) / np.pi, r.x

    def __call__(self, theta):
        return _SpectrumFn.apply(theta, self)


def _make_fn():
    import torch

    class SpectrumFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, model):
            A, x = model.solve(theta.detach().cpu().numpy())
            ctx.model = model
            ctx.x = x
            return torch.as_tensor(A, dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(ctx, grad_A):
            model = ctx.model
            g = model.solver.bilinear(model.terms.device_terms, ctx.x)          # [K, nterm]: x_k^T H_t x_k
            dA = -np.imag(g) / np.pi                                           # dA_k / dtheta_t
            grad = dA.T @ grad_A.detach().cpu().numpy().astype(np.float64)
            return torch.as_tensor(grad, dtype=grad_A.dtype, device=grad_A.device), None

    return SpectrumFn


class _Lazy:
    fn = None

    @classmethod
    def apply(cls, theta, model):
        if cls.fn is None:
            cls.fn = _make_fn()
        return cls.fn.apply(theta, model)


_SpectrumFn = _Lazy


class GreenBilinear:
    """G_ab(z_k) = a^T G(z_k) b for all shifts (complex), differentiable in theta.

    a = None means a = b: one full-mode solve, y_k = x_k.  Otherwise the
    forward pass solves for b (x_k, with a as a left vector so that a^T x_k comes
    from the projected recurrences) and for a (y_k); the backward pass forms
    y_k^T H_t x_k with kw_bilinear and returns Re(sum_k conj(g_k) dG_k/dtheta_t)
    for the incoming gradient g (PyTorch's convention for complex outputs)."""

    def __init__(self, terms, b, z, a=None, prec: str = "df64", tol: float = 1e-10, maxiter: int = 200000,
                 shift_fp32: bool = False):
        import torch

        self.terms = TermSet(terms)
        self.b = torch.as_tensor(np.asarray(b, dtype=np.float64), device="cuda")
        self.a = None if a is None else torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda")
        self.z = np.asarray(z, dtype=np.complex128)
        self.solver = kw.Solver(prec, tol=tol, maxiter=maxiter)
        self.solver.set_shift_storage(shift_fp32)
        self.rowptr = torch.as_tensor(self.terms.rowptr, device="cuda")
        self.col = torch.as_tensor(self.terms.col, device="cuda")

    def solve(self, theta):
        """Forward solves; returns (G_ab [K] complex numpy, x [K, m], y [K, m] or None)."""
        import torch

        vals = torch.as_tensor(self.terms.values(theta), device="cuda")
        self.solver.set_csr(self.rowptr, self.col, vals)
        left = None if self.a is None else self.a[None, :]
        r = self.solver.solve(self.b, self.z, left=left, full=True)
        if r.status != "KW_OK":
            raise kw.KomegaError(kw.KW_NOT_CONVERGED, f"forward solve: {r.status} after {r.iters} iterations")
        if self.a is None:
            return r.proj[:, 0].copy(), r.x, None
        ry = self.solver.solve(self.a, self.z, full=True)
        if ry.status != "KW_OK":
            raise kw.KomegaError(kw.KW_NOT_CONVERGED, f"second solve: {ry.status} after {ry.iters} iterations")
        return r.proj[:, 1].copy(), r.x, ry.x

    def __call__(self, theta):
        return _GreenLazy.apply(theta, self)


def _make_green_fn():
    import torch

    class GreenFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, model):
            G, x, y = model.solve(theta.detach().cpu().numpy())
            ctx.model = model
            ctx.x, ctx.y = x, y
            return torch.as_tensor(G, dtype=torch.complex128, device=theta.device)

        @staticmethod
        def backward(ctx, grad_G):
            model = ctx.model
            J = model.solver.bilinear(model.terms.device_terms, ctx.x, ctx.y)    # [K, nterm]: y_k^T H_t x_k
            g = grad_G.detach().cpu().numpy().astype(np.complex128)
            grad = np.real(np.conj(g) @ J)
            return torch.as_tensor(grad, dtype=torch.float64, device=grad_G.device), None

    return GreenFn


class _GreenLazy:
    fn = None

    @classmethod
    def apply(cls, theta, model):
        if cls.fn is None:
            cls.fn = _make_green_fn()
        return cls.fn.apply(theta, model)
