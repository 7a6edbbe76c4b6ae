"""Oracle: plain definitions of the shifted solution on small dense problems.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Eq. 4-5 of the Komega paper: x^(k) = G(z_k) b with G(z) = (z I - H)^{-1}
  (Eq. 2), by a dense LU solve per shift.
* Eq. 3 (spectral decomposition): G(z) = sum_j y_j y_j^T / (z - lambda_j) for
  real symmetric H, by a full eigendecomposition.  Gives a^T G(z) b
  (Eq. 1 / the G_ab of Sec. 2.2.3) without any linear solve.
"""
from __future__ import annotations

import numpy as np


def dense_solutions(Hd: np.ndarray, b: np.ndarray, z: np.ndarray) -> np.ndarray:
    """x_k = (z_k I - H)^{-1} b for every shift, [K, M] complex."""
    M = Hd.shape[0]
    eye = np.eye(M)
    return np.stack([np.linalg.solve(zk * eye - Hd, b.astype(np.complex128)) for zk in z])


def lehmann_green(Hd: np.ndarray, b: np.ndarray, z: np.ndarray, left: np.ndarray | None = None):
    """[K, L+1] values a_l^T G(z_k) b (a_0 = b) from G = sum_j y_j y_j^T / (z - lambda_j)."""
    lam, Yv = np.linalg.eigh(Hd)
    A = b[None, :] if left is None else np.vstack([b[None, :], left])
    ca = A @ Yv            # [L+1, J] components a_l . y_j
    cb = Yv.T @ b          # [J]      components y_j . b
    return np.stack([(ca * cb[None, :]) @ (1.0 / (zk - lam)) for zk in z])


def spectrum_distance(Hd: np.ndarray, z: np.ndarray) -> np.ndarray:
    """dist(z_k, spec H) = min_j |z_k - lambda_j|."""
    lam = np.linalg.eigvalsh(Hd)
    return np.array([np.min(np.abs(zk - lam)) for zk in z])
