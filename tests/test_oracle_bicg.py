"""CPU pins for the shifted BiCG and CG oracle (oracle/shifted_bicg.py; Table 1, Appendix B).

* BiCG with r~_0 = conj(b) on a complex-symmetric A = zI - H reproduces COCG:
  then r~_n = conj(r_n) at every step and r~^dagger r = r^T r.
* Shifted CG with real shifts gives, for every shift, the iterates of a plain
  textbook CG run on that shift's own system (written here from the CG
  recurrences), and seed switching does not change them beyond rounding.
* Converged BiCG on a non-Hermitian complex H and CG on a Hermitian complex H
  (real shifts) agree with the dense definition within res / sigma_min.
* Petrov-Galerkin: the BiCG residual after n steps is orthogonal (conjugated
  product) to K_n(A^dagger, b~) for every shift.
* Planted mistakes in the shadow recurrence or the inner products are caught.
"""
import sys
import types

import numpy as np
import pytest
import scipy.sparse as sp

import oracle.shifted_bicg as ob_mod
from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import workloads as w


def _anderson(L=6, seed=3):
    H = w.anderson_3d(L, 2.0, seed=seed).to_scipy()
    b = w.gaussian_unit(H.shape[0], seed + 1)
    return H, b


def _nonhermitian(m=40, seed=1):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    b = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    return A, b / np.linalg.norm(b)


def _hermitian(m=50, seed=2):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    H = (A + A.conj().T) / 2
    b = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    return H, b / np.linalg.norm(b)


@pytest.mark.parametrize("full", [True, False])
def test_bicg_with_conjugate_shadow_is_cocg(full):
    H, b = _anderson()
    left = np.stack([w.gaussian_unit(H.shape[0], 20 + i) for i in range(2)])
    z = w.shiftk_grid(-8, 8, 24, 0.05)
    rb = ob_mod.shifted_bicg(H, b, z, left=left, tol=1e-10, full=full, method="bicg")
    rc = oc.shifted_cocg(H, b, z, left=left, tol=1e-10, full=full)
    assert rb.status == rc.status == oc.STATUS_OK
    assert abs(rb.iters - rc.iters) <= 2 and rb.n_seed_switch > 0
    assert np.abs(rb.proj - rc.proj).max() <= 1e-9 * np.abs(rc.proj).max()
    n = 12                                   # before rounding differences grow: the same iterates
    rb = ob_mod.shifted_bicg(H, b, z, left=left, tol=0.0, maxiter=n, full=full, method="bicg")
    rc = oc.shifted_cocg(H, b, z, left=left, tol=0.0, maxiter=n, full=full)
    assert np.abs(rb.proj - rc.proj).max() <= 1e-12 * np.abs(rc.proj).max()


def _textbook_cg(A, b, n):
    """n steps of CG (Hermitian A, x_0 = 0), conjugated inner products."""
    x = np.zeros_like(b, dtype=np.complex128)
    r = b.astype(np.complex128)
    p = r.copy()
    rr = np.vdot(r, r)
    for _ in range(n):
        Ap = A @ p
        a = rr / np.vdot(p, Ap)
        x = x + a * p
        r = r - a * Ap
        rr_new = np.vdot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


@pytest.mark.parametrize("switch", [False, True])
@pytest.mark.parametrize("n", [1, 3, 8])
def test_cg_iterates_are_textbook_cg_per_shift(n, switch):
    H, b = _hermitian(m=30, seed=4)
    ev = np.linalg.eigvalsh(H)
    z = np.array([ev[0] - 0.5, ev[0] - 2.0, ev[-1] + 1.0, ev[-1] + 3.0], dtype=np.complex128)   # definite systems
    r = ob_mod.shifted_bicg(H, b, z, tol=0.0, maxiter=n, full=True, method="cg", seed_switch=switch)
    for k, zk in enumerate(z):
        xk = _textbook_cg(zk.real * np.eye(30) - H, b, n)
        assert np.linalg.norm(r.x[k] - xk) <= 1e-11 * np.linalg.norm(xk), (k, n)


def _dense_check(H, b, z, r, factor=2.0):
    M = b.size
    Hd = H.toarray() if sp.issparse(H) else H
    for k, zk in enumerate(z):
        A = zk * np.eye(M) - Hd
        xk = np.linalg.solve(A, b)
        smin = np.linalg.svd(A, compute_uv=False)[-1]
        assert np.linalg.norm(r.x[k] - xk) <= factor * r.final_res[k] / smin + 1e-12, k


def test_bicg_nonhermitian_matches_dense():
    A, b = _nonhermitian()
    z = np.array([2.5 + 0.3j, -2.2 + 0.5j, 0.3 + 2.0j, 3.0 - 1.0j])
    r = ob_mod.shifted_bicg(A, b, z, tol=1e-10, maxiter=400, full=True, method="bicg")
    assert r.status == oc.STATUS_OK
    _dense_check(A, b, z, r)


def test_cg_hermitian_real_shifts_matches_dense():
    H, b = _hermitian()
    ev = np.linalg.eigvalsh(H)
    z = np.concatenate([np.linspace(ev[0] - 3, ev[0] - 0.2, 4), np.linspace(ev[-1] + 0.2, ev[-1] + 3, 4)])
    r = ob_mod.shifted_bicg(H, b, z.astype(np.complex128), tol=1e-11, maxiter=400, full=True, method="cg")
    assert r.status == oc.STATUS_OK
    _dense_check(H, b, z, r)


@pytest.mark.parametrize("n", [2, 4, 7])
def test_bicg_petrov_galerkin(n):
    A, b = _nonhermitian(m=30, seed=5)
    rng = np.random.default_rng(9)
    bt = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    z = np.array([2.5 + 0.3j, -2.2 + 0.5j, 0.3 + 2.0j])
    r = ob_mod.shifted_bicg(A, b, z, tol=0.0, maxiter=n, full=True, method="bicg", btilde=bt, seed_switch=False)
    for k, zk in enumerate(z):
        Ak = zk * np.eye(30) - A
        res = b - Ak @ r.x[k]
        # K_n(A_k^dagger, b~) is spanned by (A^dagger)^i b~ for the seed's A: same space for every shift
        V = np.stack([np.linalg.matrix_power(Ak.conj().T, i) @ bt for i in range(n)], axis=1)
        Q, _ = np.linalg.qr(V)
        assert np.abs(Q.conj().T @ res).max() <= 1e-9 * np.linalg.norm(b), (k, n)


# ------------------------------------------------------------- planted mistakes
SRC = open(ob_mod.__file__).read()
MUTATIONS = {
    "shadow_alpha_not_conjugated": ("- np.conj(alpha) * qt", "- alpha * qt"),
    "shadow_c_not_conjugated": ("rt_new = (1.0 + np.conj(c)) * rt", "rt_new = (1.0 + c) * rt"),
    "shadow_product_not_adjoint": ("qt = np.conj(z[s]) * rt - Hh @ rt", "qt = np.conj(z[s]) * rt - H @ rt"),
    "unconjugated_rho": ("rho_new = np.vdot(rt_new, r_new)", "rho_new = np.dot(rt_new, r_new)"),
    "shadow_switch_scale": ("rt = rt / np.conj(pj_new)", "rt = rt / pj_new"),
}


def _mutant(name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, name
    mod = types.ModuleType("bicg_mutant_" + name)
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(SRC.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


def _pins_pass(mod):
    # BiCG with the conjugate shadow is COCG step for step (switches happen every step here)
    H, bb = _anderson()
    zz = w.shiftk_grid(-8, 8, 24, 0.05)
    with np.errstate(all="ignore"):
        rb = mod.shifted_bicg(H, bb, zz, tol=0.0, maxiter=30, full=False, method="bicg")
    rc = oc.shifted_cocg(H, bb, zz, tol=0.0, maxiter=30, full=False)
    if not np.all(np.isfinite(rb.proj)) or np.abs(rb.proj - rc.proj).max() > 1e-12 * np.abs(rc.proj).max():
        return False
    A, b = _nonhermitian(m=30, seed=7)
    z = np.array([2.5 + 0.3j, -2.2 + 0.5j, 0.3 + 2.0j, 0.2 + 0.4j])
    with np.errstate(all="ignore"):
        r = mod.shifted_bicg(A, b, z, tol=1e-10, maxiter=300, full=True, method="bicg")
    if r.status != oc.STATUS_OK or not np.all(np.isfinite(r.x)):
        return False
    for k, zk in enumerate(z):
        xk = np.linalg.solve(zk * np.eye(30) - A, b)
        if np.linalg.norm(r.x[k] - xk) > 1e-6 * np.linalg.norm(xk):
            return False
    return True


def test_pins_accept_the_oracle():
    assert _pins_pass(ob_mod)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_reject_planted_mistake(name):
    assert not _pins_pass(_mutant(name))
