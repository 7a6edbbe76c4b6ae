"""The oracle pins must catch plausible mistakes.

Each case plants one mistake (a sign, a dropped power, a wrong index, a
conjugated product, a freeze-rule slip) into a copy of the oracle's source,
loads the copy as a separate module and checks that the Galerkin / projection
/ freeze pins reject it.  The real oracle is never modified.
"""
import sys
import types

import numpy as np
import pytest

import oracle.shifted_cocg as oc_mod

SRC = open(oc_mod.__file__).read()

MUTATIONS = {
    "pi_sign": ("(1.0 + c + alpha * sigma[k]) * pi[k]", "(1.0 + c - alpha * sigma[k]) * pi[k]"),
    "beta_power": ("beta_k = ratio * ratio * beta", "beta_k = ratio * beta"),
    "conjugated_alpha_dot": ("denom = np.dot(r, q)", "denom = np.vdot(r, q)"),
    "three_term_sign": ("- alpha * q - c * r_old", "- alpha * q + c * r_old"),
    "u_index": ("U[k] = w[None, :] / pi_new_k[:, None]", "U[k] = w[None, :] / pi[k][:, None]"),
    "switch_r_old_index": ("r_old = r_old / pj_old", "r_old = r_old / pj_new"),
    "switch_beta_alpha": ("beta_over_alpha = beta_over_alpha * pj_old / pj_new",
                          "beta_over_alpha = beta_over_alpha"),
    "stale_seed_shift": ("q = z[s] * r - _matvec(H, r)", "q = z[0] * r - _matvec(H, r)"),
    "conv_iter_off_by_one": ("conv_iter[k[done]] = n + 1", "conv_iter[k[done]] = n"),
    "residual_unsquared": ("res_k = np.sqrt(nu_new) / np.abs(pi_new_k)", "res_k = nu_new / np.abs(pi_new_k)"),
    "residual_old_pi": ("res_k = np.sqrt(nu_new) / np.abs(pi_new_k)", "res_k = np.sqrt(nu_new) / np.abs(pi[k])"),
    "p_update_order": ("X[k] += alpha_k[:, None] * Pv[k]\n            Pv[k] = r_new[None, :] / pi_new_k[:, None] + beta_k[:, None] * Pv[k]",
                       "Pv[k] = r_new[None, :] / pi_new_k[:, None] + beta_k[:, None] * Pv[k]\n            X[k] += alpha_k[:, None] * Pv[k]"),
}


def _load_mutant(name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, name
    return _exec_module(f"oracle_mutant_{name}", SRC.replace(old, new))


def _exec_module(modname, source):
    mod = types.ModuleType(modname)
    sys.modules[modname] = mod  # dataclasses resolve their module through sys.modules
    try:
        exec(compile(source, f"<{modname}>", "exec"), mod.__dict__)
    finally:
        del sys.modules[modname]
    return mod


def _galerkin(Hd, b, zk, n):
    M = b.size
    V = np.zeros((M, n))
    v = b.copy()
    for i in range(n):
        V[:, i] = v
        v = Hd @ v
    Q, _ = np.linalg.qr(V)
    return Q @ np.linalg.solve(Q.T @ (zk * np.eye(M) - Hd) @ Q, Q.T @ b)


def _freeze_pin_passes(mod):
    """The freeze rule: shift k stops at the first n whose Galerkin iterate has
    true residual <= tol ||b||, keeps it, and reports that residual."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 30))
    Hd = (A + A.T) / 2
    b = rng.standard_normal(30)
    b /= np.linalg.norm(b)
    z = np.array([0.5 + 3j, -2 + 2.5j, 3 + 4j, 1 + 6j, -4 + 3.5j, 6 + 5j])
    tol = 1e-4
    with np.errstate(all="ignore"):
        r = mod.shifted_cocg(Hd, b, z, tol=tol, maxiter=30, full=True)
    Q = np.zeros((30, 30))
    v = b.copy()
    for i in range(30):
        Q[:, i] = v
        if i == 29:
            break
        u = Hd @ v
        for _ in range(2):
            u -= Q[:, :i + 1] @ (Q[:, :i + 1].T @ u)
        v = u / np.linalg.norm(u)
    for k, zk in enumerate(z):
        Ak = zk * np.eye(30) - Hd
        for n in range(1, 31):
            Qn = Q[:, :n]
            x = Qn @ np.linalg.solve(Qn.T @ Ak @ Qn, Qn.T @ b)
            t = np.linalg.norm(b - Ak @ x)
            if t <= tol:
                break
        if r.x is None or r.conv_iter[k] != n or np.linalg.norm(r.x[k] - x) > 1e-9 * np.linalg.norm(x):
            return False
        if not abs(r.final_res[k] - t) <= 1e-9 * t:
            return False
    return True


def _pins_pass(mod):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 30))
    Hd = (A + A.T) / 2
    b = rng.standard_normal(30)
    b /= np.linalg.norm(b)
    left = rng.standard_normal((2, 30))
    z = np.array([0.3 + 0.5j, -1 + 0.2j, 2 + 1j, 0.1 + 0.05j])
    for n in (2, 3, 6):
        with np.errstate(all="ignore"):
            rf = mod.shifted_cocg(Hd, b, z, left=left, tol=0.0, maxiter=n, full=True)
            rp = mod.shifted_cocg(Hd, b, z, left=left, tol=0.0, maxiter=n, full=False)
        xs = np.stack([_galerkin(Hd, b, zk, n) for zk in z])
        if rf.x is None or rf.x.shape != xs.shape or not np.all(np.isfinite(rf.x)):
            return False
        if np.abs(rf.x - xs).max() > 1e-9:
            return False
        ref = xs @ np.vstack([b, left]).T
        if rp.proj is None or np.abs(rp.proj - ref).max() > 1e-9:
            return False
    return _freeze_pin_passes(mod)


def test_unmutated_copy_passes():
    assert _pins_pass(_exec_module("oracle_copy", SRC))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name):
    assert not _pins_pass(_load_mutant(name))
