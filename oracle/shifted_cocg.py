"""Oracle: shifted COCG for (z_k I - H) x^(k) = b, plain FP64 on the CPU.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference that the
CUDA path is checked against.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import it; the product path never does.
It shares no code with the CUDA path.

What it computes (Komega paper, Sec. 2.2 and Appendix A):

* Seed system A x = b with A = z_s I - H (Eq. 6; sigma_k = z_k - z_s).
* Three-term residual recurrence (Eq. 16) with the alpha formula (Eq. 17),
  starting from beta_{-1}/alpha_{-1} = 0, r_0 = b, r_{-1} = 0.
* COCG (Appendix A): every inner product of the CG formulas (Eqs. 10, 17) is
  the unconjugated x^T y.  The residual norm used for convergence stays the
  ordinary 2-norm of Eq. 7.
* Collinear residuals r_n^sigma = r_n / pi_n^sigma (Eq. 19) with the pi
  recurrence (Eq. 20), pi_0 = pi_{-1} = 1.
* Shifted alpha, beta, x, p recurrences (Eqs. 21-24), x_0 = 0, p_0 = b.
* Projected mode (Eqs. 25-26, Sec. 2.2.3): y = P x, u_0 = P b, with the rows
  of P the left vectors a_l; the index reading of Eq. 26 used here is
  u_{n+1} = (1/pi_{n+1}) P r_{n+1} + beta_n^sigma u_n (the form that matches
  Eq. 24 term by term).
* Seed switching after every update (Sec. 2.2.4): switch to the active shift
  with the smallest |pi_{n+1}| when it is below the current seed's (= 1).
  Reading used for the formulas (the paper cites them from elsewhere):
  r_{n+1} <- r_{n+1}/pi^j_{n+1}, r_n <- r_n/pi^j_n,
  rho_{n+1} <- r_{n+1}^T r_{n+1},
  beta_n/alpha_n <- (beta_n/alpha_n) pi^j_n / pi^j_{n+1},
  pi^k_{n+1} <- pi^k_{n+1}/pi^j_{n+1}, pi^k_n <- pi^k_n/pi^j_n (the new
  seed's factors set to exactly 1), sigma_k <- z_k - z_j.
  The shifted x, p (or y, u) are untouched.
* Convergence per shift (Sec. 3.2.2, convfactor criterion read as relative
  and per shift): res_k = ||r_{n+1}||_2 / |pi^k_{n+1}| <= tol * ||b||_2.
  A shift that meets it is frozen: no further update of x, p, y, u or pi.

Arithmetic: complex128 throughout.  The sparse product H @ r and the dot
products are library primitives (scipy.sparse, numpy).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

STATUS_OK = "ok"
STATUS_NOT_CONVERGED = "not_converged"
STATUS_BREAKDOWN = "breakdown"
STATUS_NONFINITE = "nonfinite"


@dataclass
class OracleResult:
    proj: np.ndarray                 # [K, L+1] complex: column 0 = b^T x_k, then a_l^T x_k
    x: np.ndarray | None             # [K, M] complex (full mode) else None
    iters: int                       # seed iterations performed (= matrix-vector products)
    conv_iter: np.ndarray            # [K] iteration at which shift k was frozen, -1 if never
    final_res: np.ndarray            # [K] last residual estimate ||r||/|pi|
    hist: np.ndarray                 # [n_rec, K] residual estimates every hist_stride iterations
    n_seed_switch: int
    status: str
    seeds: list = field(default_factory=list)       # seed index after each iteration
    alpha: list = field(default_factory=list)       # seed alpha_n per iteration
    beta: list = field(default_factory=list)        # seed beta_n per iteration
    updates: int = 0                 # sum over iterations of the number of active shifts
    log: "KrylovLog | None" = None   # per-iteration record for recalculation (log=True)


@dataclass
class KrylovLog:
    """What a run keeps so the projections can be recomputed at other shifts
    without matrix-vector products (Sec. 3.3 (iv)): per iteration n the seed
    shift used, the seed's alpha_n, c_n, beta_n, ||r_{n+1}||^2, the projected
    residual P r_{n+1} (before any seed switch of that iteration) and the
    switch factors pi^j_{n+1}, pi^j_n of the new seed j (1, 1 when the seed
    was kept).  w0 = P r_0 = P b; thresh = tol * ||b||."""
    zs: np.ndarray        # [n] complex
    alpha: np.ndarray     # [n] complex
    c: np.ndarray         # [n] complex
    beta: np.ndarray      # [n] complex
    nu: np.ndarray        # [n] real
    pj1: np.ndarray       # [n] complex
    pj0: np.ndarray       # [n] complex
    w: np.ndarray         # [n, L+1] complex
    w0: np.ndarray        # [L+1] complex
    thresh: float


def _matvec(H, v):
    return H @ v


def shifted_cocg(H, b, z, left=None, tol=1e-10, maxiter=100000, full=True,
                 seed_switch=True, hist_stride=1, seed0=0, log=False):
    """Solve (z_k I - H) x_k = b for all shifts z by shifted COCG.

    H: real symmetric matrix supporting ``H @ v`` (scipy sparse or dense).
    b: real [M].  z: complex [K].  left: real [L, M] or None.
    full: keep the x_k (Eqs. 23-24); otherwise only the projections (Eqs. 25-26).
    log: also return the KrylovLog of the run (for ``oracle.recalc``).
    Returns an OracleResult; proj[:, 0] is b^T x_k in both modes.
    """
    b = np.asarray(b, dtype=np.float64)
    z = np.asarray(z, dtype=np.complex128)
    M = b.size
    K = z.size
    P = b[None, :] if left is None else np.vstack([b[None, :], np.asarray(left, dtype=np.float64)])
    norm_b = np.sqrt(np.dot(b, b))
    thresh = tol * norm_b

    # Seed index s and shifts sigma_k = z_k - z_s (Eq. 6).
    s = seed0
    sigma = z - z[s]

    # Seed vectors: r_n, r_{n-1} (three-vector memory scheme, Sec. 2.2.3).
    r = b.astype(np.complex128)
    r_old = np.zeros(M, dtype=np.complex128)
    rho = np.dot(r, r)                     # Eq. 10 with the COCG product
    beta_over_alpha = 0.0 + 0.0j           # beta_{-1}/alpha_{-1} = 0

    # Collinearity factors pi_n, pi_{n-1} (Eq. 20 initialisation).
    pi = np.ones(K, dtype=np.complex128)
    pi_old = np.ones(K, dtype=np.complex128)
    active = np.ones(K, dtype=bool)

    if full:
        X = np.zeros((K, M), dtype=np.complex128)
        Pv = np.tile(b.astype(np.complex128), (K, 1))          # p_0 = b
    else:
        Y = np.zeros((K, P.shape[0]), dtype=np.complex128)
        U = np.tile((P @ b).astype(np.complex128), (K, 1))     # u_0 = P b

    conv_iter = np.full(K, -1, dtype=np.int64)
    final_res = np.full(K, np.inf)
    hist = []
    res = OracleResult(proj=None, x=None, iters=0, conv_iter=conv_iter, final_res=final_res,
                       hist=None, n_seed_switch=0, status=STATUS_NOT_CONVERGED)

    lg = {key: [] for key in ("zs", "alpha", "c", "beta", "nu", "pj1", "pj0", "w")}

    n = 0
    while n < maxiter and active.any():
        # --- seed system: q = A r_n, alpha_n (Eq. 17), three-term update (Eq. 16)
        q = z[s] * r - _matvec(H, r)
        if rho == 0:
            res.status = STATUS_BREAKDOWN
            break
        denom = np.dot(r, q) - beta_over_alpha * rho
        if denom == 0:
            res.status = STATUS_BREAKDOWN
            break
        alpha = rho / denom
        c = alpha * beta_over_alpha
        r_new = (1.0 + c) * r - alpha * q - c * r_old
        rho_new = np.dot(r_new, r_new)
        beta = rho_new / rho
        nu_new = np.real(np.vdot(r_new, r_new))              # ||r_{n+1}||^2 (Eq. 7 norm)
        if not (np.isfinite(alpha) and np.isfinite(beta) and np.isfinite(nu_new)):
            res.status = STATUS_NONFINITE
            break

        if log:
            lg["zs"].append(z[s])
            lg["alpha"].append(alpha)
            lg["c"].append(c)
            lg["beta"].append(beta)
            lg["nu"].append(nu_new)
            lg["w"].append(P @ r_new)
            lg["pj1"].append(1.0 + 0.0j)
            lg["pj0"].append(1.0 + 0.0j)

        # --- shifted systems (Eqs. 20-26), active shifts only
        k = np.nonzero(active)[0]
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
            w = P @ r_new                                      # P r_{n+1}
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

        # --- rotate the seed recurrence
        r_old = r
        r = r_new
        rho = rho_new
        beta_over_alpha = beta / alpha
        res.alpha.append(alpha)
        res.beta.append(beta)
        n += 1
        if hist_stride and n % hist_stride == 0:
            hist.append(final_res.copy())

        # --- seed switching (Sec. 2.2.4), after every update
        if seed_switch and active.any():
            ka = np.nonzero(active)[0]
            mag2 = pi[ka].real ** 2 + pi[ka].imag ** 2
            j = ka[np.argmin(mag2)]                            # lowest index on ties
            if mag2.min() < 1.0:
                pj_new, pj_old = pi[j], pi_old[j]
                if log:
                    lg["pj1"][-1] = pj_new
                    lg["pj0"][-1] = pj_old
                r = r / pj_new
                r_old = r_old / pj_old
                rho = np.dot(r, r)
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
    if log:
        n_log = n                                              # completed iterations only
        cplx = lambda key: np.array(lg[key][:n_log], dtype=np.complex128).reshape(n_log)
        res.log = KrylovLog(zs=cplx("zs"), alpha=cplx("alpha"), c=cplx("c"), beta=cplx("beta"),
                            nu=np.array(lg["nu"][:n_log], dtype=np.float64).reshape(n_log), pj1=cplx("pj1"),
                            pj0=cplx("pj0"),
                            w=np.array(lg["w"][:n_log], dtype=np.complex128).reshape(n_log, P.shape[0]),
                            w0=(P @ b).astype(np.complex128), thresh=float(thresh))
    return res


def csr_matvec(rowptr, col, val, v):
    """Plain CSR product y = H v, one row at a time (for independent residual checks)."""
    import scipy.sparse as sp

    m = rowptr.size - 1
    return sp.csr_matrix((val, col, rowptr), shape=(m, m)) @ v


def true_residuals(H, b, z, X):
    """||b - (z_k I - H) x_k||_2 for every shift (Eq. 7 with x_k given)."""
    out = np.empty(z.size)
    for k in range(z.size):
        rk = b - (z[k] * X[k] - H @ X[k])
        out[k] = np.sqrt(np.real(np.vdot(rk, rk)))
    return out
