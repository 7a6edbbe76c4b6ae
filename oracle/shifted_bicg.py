"""Oracle: shifted BiCG and shifted CG for (z_k I - H) x^(k) = b, plain FP64.

TEST INFRASTRUCTURE ONLY (see the package header): only the tests, the smoke
check and the CPU-baseline leg of the benchmark import it.

What it computes (Komega paper, Table 1 and Appendix B):

* Table 1 selects the solver by the type of A + sigma I: CG for real
  symmetric or Hermitian (real shifts), COCG for complex symmetric, BiCG
  otherwise.  ``shifted_cocg`` is the COCG oracle; this module holds the other
  two.
* BiCG (Appendix B): besides r_n it carries the shadow residual r~_n of the
  adjoint seed system, with rho_n = r~_n^dagger r_n,
    alpha_n = rho_n / (r~_n^dagger A r_n - (beta_{n-1}/alpha_{n-1}) rho_n),
    r_{n+1}  = (1 + c_n - alpha_n A) r_n - c_n r_{n-1},
    r~_{n+1} = (1 + c_n^* - alpha_n^* A^dagger) r~_n - c_n^* r~_{n-1},
    beta_n = rho_{n+1} / rho_n, c_n = alpha_n beta_{n-1}/alpha_{n-1},
  with A = z_s I - H, r_0 = b, r~_0 = b~ (any vector not orthogonal to b).
* CG: the same recurrence with the shadow equal to the residual itself
  (r~_n = r_n, so rho_n = ||r_n||^2) for Hermitian A; Table 1 uses it with
  real shifts, where every scalar is real.
* Shifted systems: the residuals stay collinear, r_n^sigma = r_n / pi_n^sigma,
  and x, p (or the projections y, u) follow Eqs. 20-26 exactly as in COCG.
* Seed switching (Sec. 2.2.4) as in the COCG oracle; the shadow residuals of
  the new seed are r~ / (pi^j)^* (their shifted systems use sigma^*), so rho
  scales by 1/(pi^j)^2 as in COCG.

H: anything supporting ``H @ v`` (complex allowed); ``H.conj().T @ v`` is used
for A^dagger (scipy sparse and numpy arrays provide it).
"""
from __future__ import annotations

import numpy as np

from oracle.shifted_cocg import (OracleResult, STATUS_BREAKDOWN, STATUS_NONFINITE, STATUS_NOT_CONVERGED,
                                 STATUS_OK)


def shifted_bicg(H, b, z, left=None, tol=1e-10, maxiter=100000, full=True, seed_switch=True, method="bicg",
                 btilde=None, seed0=0):
    """Shifted BiCG (method='bicg') or shifted CG (method='cg') for all shifts z.

    b: real or complex [M].  btilde: BiCG shadow start (default conj(b)).
    Returns an OracleResult; proj[:, 0] is b^T x_k (unconjugated, as in COCG),
    then a_l^T x_k for real left vectors a_l."""
    if method not in ("bicg", "cg"):
        raise ValueError("method must be 'bicg' or 'cg'")
    b = np.asarray(b)
    z = np.asarray(z, dtype=np.complex128)
    M, K = b.size, z.size
    Hh = H.conj().T
    P = b[None, :] if left is None else np.vstack([b[None, :], np.asarray(left, dtype=np.float64)])
    thresh = tol * np.linalg.norm(b)
    s = seed0
    sigma = z - z[s]

    r = b.astype(np.complex128)
    r_old = np.zeros(M, dtype=np.complex128)
    if method == "bicg":
        rt = (np.conj(b) if btilde is None else np.asarray(btilde)).astype(np.complex128)
        rt_old = np.zeros(M, dtype=np.complex128)
        rho = np.vdot(rt, r)
    else:
        rho = np.vdot(r, r)
    beta_over_alpha = 0.0 + 0.0j

    pi = np.ones(K, dtype=np.complex128)
    pi_old = np.ones(K, dtype=np.complex128)
    active = np.ones(K, dtype=bool)
    if full:
        X = np.zeros((K, M), dtype=np.complex128)
        Pv = np.tile(r, (K, 1))
    else:
        Y = np.zeros((K, P.shape[0]), dtype=np.complex128)
        U = np.tile((P @ r).astype(np.complex128), (K, 1))
    conv_iter = np.full(K, -1, dtype=np.int64)
    final_res = np.full(K, np.inf)
    hist = []
    res = OracleResult(proj=None, x=None, iters=0, conv_iter=conv_iter, final_res=final_res, hist=None,
                       n_seed_switch=0, status=STATUS_NOT_CONVERGED)
    n = 0
    while n < maxiter and active.any():
        q = z[s] * r - H @ r                                   # A r_n
        shadow = rt if method == "bicg" else r
        if rho == 0:
            res.status = STATUS_BREAKDOWN
            break
        denom = np.vdot(shadow, q) - beta_over_alpha * rho    # r~^dagger A r - (beta/alpha) rho
        if denom == 0:
            res.status = STATUS_BREAKDOWN
            break
        alpha = rho / denom
        c = alpha * beta_over_alpha
        r_new = (1.0 + c) * r - alpha * q - c * r_old
        if method == "bicg":
            qt = np.conj(z[s]) * rt - Hh @ rt                   # A^dagger r~_n
            rt_new = (1.0 + np.conj(c)) * rt - np.conj(alpha) * qt - np.conj(c) * rt_old
            rho_new = np.vdot(rt_new, r_new)
        else:
            rho_new = np.vdot(r_new, r_new)
        beta = rho_new / rho
        nu_new = np.real(np.vdot(r_new, r_new))
        if not (np.isfinite(alpha) and np.isfinite(beta) and np.isfinite(nu_new)):
            res.status = STATUS_NONFINITE
            break

        k = np.nonzero(active)[0]                              # Eqs. 20-26, as in COCG
        pi_new_k = (1.0 + c + alpha * sigma[k]) * pi[k] - c * pi_old[k]
        if np.any(pi_new_k == 0):
            res.status = STATUS_BREAKDOWN
            break
        ratio = pi[k] / pi_new_k
        alpha_k = ratio * alpha
        beta_k = ratio * ratio * beta
        if full:
            X[k] += alpha_k[:, None] * Pv[k]
            Pv[k] = r_new[None, :] / pi_new_k[:, None] + beta_k[:, None] * Pv[k]
        else:
            w = P @ r_new
            Y[k] += alpha_k[:, None] * U[k]
            U[k] = w[None, :] / pi_new_k[:, None] + beta_k[:, None] * U[k]
        res_k = np.sqrt(nu_new) / np.abs(pi_new_k)
        final_res[k] = res_k
        res.updates += k.size
        pi_old[k] = pi[k]
        pi[k] = pi_new_k
        done = res_k <= thresh
        conv_iter[k[done]] = n + 1
        active[k[done]] = False

        r_old, r = r, r_new
        if method == "bicg":
            rt_old, rt = rt, rt_new
        rho = rho_new
        beta_over_alpha = beta / alpha
        res.alpha.append(alpha)
        res.beta.append(beta)
        n += 1
        hist.append(final_res.copy())

        if seed_switch and active.any():
            ka = np.nonzero(active)[0]
            mag2 = pi[ka].real ** 2 + pi[ka].imag ** 2
            j = ka[np.argmin(mag2)]
            if mag2.min() < 1.0:
                pj_new, pj_old = pi[j], pi_old[j]
                r = r / pj_new
                r_old = r_old / pj_old
                if method == "bicg":
                    rt = rt / np.conj(pj_new)
                    rt_old = rt_old / np.conj(pj_old)
                    rho = np.vdot(rt, r)
                else:
                    rho = np.vdot(r, r)
                beta_over_alpha = beta_over_alpha * pj_old / pj_new
                pi[active] = pi[active] / pj_new
                pi_old[active] = pi_old[active] / pj_old
                pi[j] = 1.0
                pi_old[j] = 1.0
                s = j
                sigma = z - z[s]
                res.n_seed_switch += 1
        res.seeds.append(s)

    if res.status == STATUS_NOT_CONVERGED and not active.any():
        res.status = STATUS_OK
    res.iters = n
    if full:
        res.x = X
        res.proj = X @ P.T
    else:
        res.proj = Y
    res.hist = np.array(hist).reshape(-1, K)
    return res
