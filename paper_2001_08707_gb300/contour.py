"""Contour-integral eigensolver on top of the shifted solver (Sec. 4.1 of the
Komega paper: the Sakurai-Sugiura method with Krylov-type moments).

For a circle Gamma: z_j = gamma + rho exp[2 pi i (j + 1/2) / N_z], j < N_z, and
N_l random vectors phi_l, the shifted solves x_{j,l} = (z_j I - H)^{-1} phi_l
give the moments

    s_{k,l} = (1/2 pi i) oint (z - gamma)^k (z I - H)^{-1} phi_l dz
            ~ (1/N_z) sum_j (z_j - gamma)^{k+1} x_{j,l}     (trapezoid rule on the circle),

which span the eigenvectors with eigenvalues inside Gamma.  Moment k is scaled
by rho^-k (same span, better conditioning).  The SVD of
S = [s_{0,0} .. s_{N_k-1,0}, s_{0,1}, ...] keeps the left singular vectors whose
singular values exceed sv_cut times the largest, and the eigenvalues of the
projected matrix U^dagger H U inside Gamma are returned.

The shifted solves are the hot path and run through ``solve_fn``; with the
CUDA solver (``gpu_moments_fn``) the moments are also formed on the device
(kw_shift_combine), so only the N_k moment vectors of each right-hand side, not
its N_z solutions, reach the host.  The SVD and the small projected eigenproblem
are dense host work.
"""
from __future__ import annotations

import numpy as np


def circle_points(gamma: float, rho: float, nz: int) -> np.ndarray:
    j = np.arange(nz, dtype=np.float64)
    return gamma + rho * np.exp(2j * np.pi * (j + 0.5) / nz)


def moment_weights(z: np.ndarray, gamma: float, rho: float, nk: int) -> np.ndarray:
    """[nk, N_z] weights: moment k = sum_j W[k, j] x_j with W[k, j] = (z_j - gamma)/N_z ((z_j - gamma)/rho)^k."""
    w = (z - gamma) / z.size                       # quadrature weight (z_j - gamma) / N_z
    t = (z - gamma) / rho
    return np.stack([w * t ** k for k in range(nk)])


def moments(X: np.ndarray, z: np.ndarray, gamma: float, rho: float, nk: int) -> np.ndarray:
    """[nk, M] moments of one right-hand side from its solutions X [N_z, M]."""
    return moment_weights(z, gamma, rho, nk) @ X


def ss_eigs(solve_fn, H, m: int, gamma: float, rho: float, nz: int, nk: int, nl: int, seed: int = 12,
            sv_cut: float = 1e-3, moments_fn=None):
    """Eigenvalues of H inside the circle (gamma, rho).

    solve_fn(phi, z) -> X [len(z), m] complex solutions of (z_j I - H) x = phi;
    or moments_fn(phi, z, W) -> [nk, m] moments W X formed where X lives (then
    solve_fn is not called).
    H: anything with H @ V for a dense [m, r] block (scipy sparse works).
    Returns (eigenvalues inside Gamma ascending, singular values of S)."""
    z = circle_points(gamma, rho, nz)
    W = moment_weights(z, gamma, rho, nk)
    rng = np.random.default_rng(seed)
    cols = []
    for _ in range(nl):
        phi = rng.standard_normal(m)
        phi /= np.linalg.norm(phi)
        cols.append(moments_fn(phi, z, W) if moments_fn is not None else W @ solve_fn(phi, z))
    S = np.concatenate(cols, axis=0).T            # [m, nk * nl]
    U, sv, _ = np.linalg.svd(S, full_matrices=False)
    keep = sv > sv_cut * sv[0]
    Uk = U[:, keep]
    Ht = Uk.conj().T @ (H @ Uk)
    ev = np.linalg.eigvals(Ht)
    ev = ev[np.abs(ev - gamma) < rho]
    return np.sort(ev.real), sv


def gpu_solve_fn(H, prec: str = "df64", tol: float = 1e-12, maxiter: int = 100000):
    """A solve_fn backed by the CUDA solver (full mode)."""
    from paper_2001_08707_gb300 import komega as kw

    s = kw.Solver(prec, tol=tol, maxiter=maxiter)
    s.set_csr(H.rowptr, H.col, H.val)

    def solve(phi, z):
        r = s.solve(phi, z, full=True)
        if r.status != "KW_OK":
            raise kw.KomegaError(kw.KW_NOT_CONVERGED, f"contour solve: {r.status}")
        return r.x.cpu().numpy().astype(np.complex128)

    return solve


def gpu_moments_fn(H, prec: str = "df64", tol: float = 1e-12, maxiter: int = 100000, shift_fp32: bool = False):
    """A moments_fn backed by the CUDA solver: full-mode solves on the device (x
    complex FP32 with shift_fp32), the moments W X formed there by
    kw_shift_combine; only the [nk, m] moments are copied to the host."""
    from paper_2001_08707_gb300 import komega as kw

    s = kw.Solver(prec, tol=tol, maxiter=maxiter)
    s.set_csr(H.rowptr, H.col, H.val)
    s.set_shift_storage(shift_fp32)

    def moments_fn(phi, z, W):
        r = s.solve(phi, z, full=True)
        if r.status != "KW_OK":
            raise kw.KomegaError(kw.KW_NOT_CONVERGED, f"contour solve: {r.status}")
        return s.shift_combine(r.x, W).cpu().numpy()

    return moments_fn
