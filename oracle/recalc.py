"""Oracle: recalculation at new shifts from a logged run (Sec. 3.3 (iv)).

TEST INFRASTRUCTURE ONLY (see the package header): only the tests, the smoke
check and the CPU-baseline leg of the benchmark import it.

A finished shifted COCG run leaves, per iteration n, the seed scalars
alpha_n, c_n, beta_n, the seed shift z_s(n), ||r_{n+1}||^2, the projected
residual P r_{n+1} and the seed-switch factors (``KrylovLog``).  For a shift
z that was not in the run, the collinearity factor pi_n^z obeys the same
recurrence as every other shift (Eq. 20, sigma = z - z_s(n)), and its
alpha^z, beta^z follow from Eqs. 21-22; the projections y = P x^z then come
from Eqs. 25-26, with u_0 = P b.  No product with H is needed.  Steps, in the
order of one iteration of the run they replay:

1. pi_{n+1} = (1 + c_n + alpha_n (z - z_s(n))) pi_n - c_n pi_{n-1}      (Eq. 20)
2. alpha^z = (pi_n/pi_{n+1}) alpha_n, beta^z = (pi_n/pi_{n+1})^2 beta_n (Eqs. 21-22)
3. y += alpha^z u;  u = P r_{n+1} / pi_{n+1} + beta^z u                  (Eqs. 25-26)
4. res = ||r_{n+1}|| / |pi_{n+1}|; freeze the shift when res <= thresh.
5. If the run switched seed after iteration n (factors pi^j_{n+1}, pi^j_n),
   divide pi_{n+1} and pi_n of every still-active shift by them (Sec. 2.2.4).

A shift still active after the last logged iteration is reported as not
converged, with its last iterate.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class RecalcResult:
    proj: np.ndarray        # [K, L+1] complex: b^T x, then a_l^T x at the new shifts
    conv_iter: np.ndarray   # [K] iteration at which the shift froze, -1 if never
    final_res: np.ndarray   # [K] last residual estimate ||r_{n+1}|| / |pi_{n+1}|
    converged: bool         # every shift froze within the logged iterations


def recalc(log, z, thresh=None):
    """Projections at shifts z from a KrylovLog (see the module docstring).

    thresh: absolute residual threshold (default: the logged run's tol*||b||)."""
    z = np.asarray(z, dtype=np.complex128)
    K = z.size
    thr = log.thresh if thresh is None else float(thresh)
    n_iter = log.alpha.size
    pi = np.ones(K, dtype=np.complex128)
    pi_old = np.ones(K, dtype=np.complex128)
    active = np.ones(K, dtype=bool)
    Y = np.zeros((K, log.w0.size), dtype=np.complex128)
    U = np.tile(log.w0, (K, 1))
    conv_iter = np.full(K, -1, dtype=np.int64)
    final_res = np.full(K, np.inf)
    for n in range(n_iter):
        if not active.any():
            break
        k = np.nonzero(active)[0]
        alpha, c, beta = log.alpha[n], log.c[n], log.beta[n]
        pi_new = (1.0 + c + alpha * (z[k] - log.zs[n])) * pi[k] - c * pi_old[k]
        ratio = pi[k] / pi_new
        alpha_k = ratio * alpha
        beta_k = ratio * ratio * beta
        Y[k] += alpha_k[:, None] * U[k]
        U[k] = log.w[n][None, :] / pi_new[:, None] + beta_k[:, None] * U[k]
        res = np.sqrt(log.nu[n]) / np.abs(pi_new)
        final_res[k] = res
        pi_old[k] = pi[k]
        pi[k] = pi_new
        done = res <= thr
        conv_iter[k[done]] = n + 1
        active[k[done]] = False
        if log.pj1[n] != 1.0 or log.pj0[n] != 1.0:
            pi[active] = pi[active] / log.pj1[n]
            pi_old[active] = pi_old[active] / log.pj0[n]
    return RecalcResult(proj=Y, conv_iter=conv_iter, final_res=final_res, converged=not active.any())
