"""Oracle: spectrum of H(theta) = sum_m theta_m H_m and its parameter gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A_k(theta) = -(1/pi) Im b^T G(z_k) b with G(z) = (z I - H)^{-1} (Eq. 2) and
x_k = G(z_k) b (Eq. 4-5).  Differentiating G (zI - H) = I gives
dG/dtheta_m = G H_m G; G is complex symmetric (H real symmetric), so
b^T G H_m G b = x_k^T H_m x_k (unconjugated) and

    dA_k/dtheta_m = -(1/pi) Im(x_k^T H_m x_k).

For the quadratic loss L = 1/2 sum_k (A_k - A*_k)^2 the gradient is
dL/dtheta_m = sum_k (A_k - A*_k) dA_k/dtheta_m.  x_k comes from the oracle's
shifted COCG in full mode; the bilinear forms are plain sparse products.
"""
from __future__ import annotations

import numpy as np

from oracle.shifted_cocg import shifted_cocg


def assemble(terms, theta):
    """H(theta) = sum_m theta_m H_m (scipy sparse terms)."""
    H = None
    for t, Hm in zip(theta, terms):
        H = t * Hm if H is None else H + t * Hm
    return H.tocsr()


def spectrum(terms, theta, b, z, tol=1e-12, maxiter=100000):
    r = shifted_cocg(assemble(terms, theta), b, z, tol=tol, full=True, maxiter=maxiter)
    return -np.imag(r.proj[:, 0]) / np.pi, r


def spectrum_and_gradient(terms, theta, b, z, target, tol=1e-12, maxiter=100000):
    """Returns (A, loss, dL/dtheta, dA/dtheta [K, nterm])."""
    A, r = spectrum(terms, theta, b, z, tol, maxiter)
    X = r.x
    dA = np.empty((z.size, len(terms)))
    for m, Hm in enumerate(terms):
        HX = (Hm @ X.T).T                              # rows: H_m x_k
        dA[:, m] = -np.imag(np.sum(X * HX, axis=1)) / np.pi
    res = A - target
    return A, 0.5 * float(res @ res), dA.T @ res, dA


def green_and_gradient(terms, theta, a, b, z, tol=1e-12, maxiter=100000):
    """G_ab(z_k) = a^T G(z_k) b for every shift and its parameter derivative
    dG_ab/dtheta_m = y_k^T H_m x_k with x_k = G(z_k) b and y_k = G(z_k) a (Eq. 2:
    dG/dtheta_m = G H_m G, and a^T G = (G^T a)^T = (G a)^T for complex symmetric
    G).  Returns (G_ab [K], dG [K, nterm]); a is b gives the single-solve case."""
    H = assemble(terms, theta)
    rx = shifted_cocg(H, b, z, tol=tol, full=True, maxiter=maxiter)
    X = rx.x
    Y = X if a is b else shifted_cocg(H, a, z, tol=tol, full=True, maxiter=maxiter).x
    G = np.sum(X * a[None, :], axis=1)                 # a^T x_k, unconjugated
    dG = np.empty((z.size, len(terms)), dtype=np.complex128)
    for m, Hm in enumerate(terms):
        HX = (Hm @ X.T).T
        dG[:, m] = np.sum(Y * HX, axis=1)
    return G, dG
