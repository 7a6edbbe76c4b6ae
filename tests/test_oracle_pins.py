"""CPU pins for the oracle: each check is fixed by the paper or by mathematics,
not by re-running the oracle's own formulas.

* Galerkin brute force: after n steps the COCG iterate of every shift is the
  unique x in K_n(H, b) with V^T (b - (z I - H) x) = 0 (Appendix A: r_n is
  orthogonal to the complex conjugate of K_n), shift by shift, independent of
  seed switching (Eq. 9 and Eq. 19).
* SPD special case: real shifts above the spectrum make z I - H symmetric
  positive definite; the iterates must equal scipy's textbook CG iterates.
* Converged solutions: dense LU (Eq. 4-5) and the spectral sum (Eq. 3).
* Freezing (Eq. 7 with Eq. 19): a shift stops at the first iteration whose
  true residual ||b - (z I - H) x_n|| of the Galerkin iterate is <= tol ||b||,
  keeps that iterate, and reports that residual.
* Sum rule, large-|z| moments, polarization identity (Sec. 3.2.2),
  degenerate inputs with closed forms.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import dense
from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import workloads as w


def _random_symmetric(M, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, M))
    Hd = (A + A.T) / 2
    b = rng.standard_normal(M)
    return Hd, b / np.linalg.norm(b)


def _galerkin(Hd, b, zk, n):
    """x in K_n(H, b) with V^T r = 0, built from an orthonormal Krylov basis."""
    M = b.size
    V = np.zeros((M, n))
    v = b.copy()
    for i in range(n):
        V[:, i] = v
        v = Hd @ v
    Q, _ = np.linalg.qr(V)
    Ak = zk * np.eye(M) - Hd
    return Q @ np.linalg.solve(Q.T @ Ak @ Q, Q.T @ b)


Z5 = np.array([0.3 + 0.5j, -1 + 0.2j, 2 + 1j, 0.1 + 0.05j, 5 + 0.01j])


@pytest.mark.parametrize("switch", [True, False])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 9])
def test_iterates_equal_galerkin(n, switch):
    Hd, b = _random_symmetric(40, 1)
    r = oc.shifted_cocg(Hd, b, Z5, tol=0.0, maxiter=n, full=True, seed_switch=switch)
    assert r.iters == n
    for k, zk in enumerate(Z5):
        xg = _galerkin(Hd, b, zk, n)
        assert np.linalg.norm(r.x[k] - xg) <= 1e-11 * np.linalg.norm(xg)


@pytest.mark.parametrize("switch", [True, False])
@pytest.mark.parametrize("n", [2, 5, 12])
def test_galerkin_error_identity_of_the_spectrum(n, switch):
    """COCG's error in b^T x: with G = (zI - H)^{-1} complex symmetric and the
    iterate x_n in K_n with V^T r_n = 0, b^T G b - b^T x_n = x*^T r_n =
    (G r_n)^T r_n = r_n^T G r_n, where r_n = b - (zI - H) x_n is the true
    residual of the shift (Appendix A; Eq. 19 makes it the seed residual over
    pi_n).  Checked against a dense inverse for every shift, with and without
    seed switching."""
    Hd, b = _random_symmetric(50, 4)
    r = oc.shifted_cocg(Hd, b, Z5, tol=0.0, maxiter=n, full=True, seed_switch=switch)
    assert r.iters == n
    for k, zk in enumerate(Z5):
        G = np.linalg.inv(zk * np.eye(b.size) - Hd)
        x = r.x[k]
        rn = b - (zk * x - Hd @ x)
        lhs = b @ G @ b - b @ x
        rhs = rn @ G @ rn
        assert abs(lhs - rhs) <= 1e-9 * abs(lhs) + 1e-13 * abs(b @ G @ b), (k, lhs, rhs)


@pytest.mark.parametrize("seed0", [0, 2, 4])
def test_iterates_independent_of_initial_seed(seed0):
    Hd, b = _random_symmetric(30, 2)
    n = 6
    r = oc.shifted_cocg(Hd, b, Z5, tol=0.0, maxiter=n, full=True, seed_switch=False, seed0=seed0)
    for k, zk in enumerate(Z5):
        xg = _galerkin(Hd, b, zk, n)
        assert np.linalg.norm(r.x[k] - xg) <= 1e-11 * np.linalg.norm(xg)


def test_projected_iterates_equal_projection_of_full():
    """Eqs. 25-26 (with the u_{n+1} index reading) give P x_n at every n."""
    Hd, b = _random_symmetric(35, 3)
    left = np.random.default_rng(9).standard_normal((3, 35))
    for n in (1, 2, 4, 7):
        rf = oc.shifted_cocg(Hd, b, Z5, left=left, tol=0.0, maxiter=n, full=True)
        rp = oc.shifted_cocg(Hd, b, Z5, left=left, tol=0.0, maxiter=n, full=False)
        xs = np.stack([_galerkin(Hd, b, zk, n) for zk in Z5])
        P = np.vstack([b, left])
        ref = xs @ P.T
        np.testing.assert_allclose(rp.proj, ref, atol=1e-11 * np.abs(ref).max())
        np.testing.assert_allclose(rf.proj, ref, atol=1e-11 * np.abs(ref).max())


def test_spd_shifts_match_textbook_cg():
    """Real shifts above the spectrum: z I - H is SPD and shifted COCG reduces to CG."""
    H = w.anderson_3d(5, 2.0, seed=4).to_scipy()
    b = w.gaussian_unit(H.shape[0], 4)
    z = np.array([7.5 + 0j, 9.0 + 0j, 12.0 + 0j])
    for n in (3, 8, 15):
        r = oc.shifted_cocg(H, b, z, tol=0.0, maxiter=n, full=True)
        for k, zk in enumerate(z):
            A = zk.real * sp.eye(H.shape[0]) - H
            its = []
            spla.cg(A, b, x0=np.zeros_like(b), rtol=1e-300, atol=0.0, maxiter=n,
                    callback=lambda xk: its.append(xk.copy()))
            assert len(its) == n
            np.testing.assert_allclose(r.x[k].real, its[-1], atol=1e-12)
            assert np.abs(r.x[k].imag).max() == 0.0


def test_converged_matches_dense_and_lehmann():
    p = w.anderson_small(L=6, K=24, delta=0.05, tol=1e-11)
    H = p.H.to_scipy()
    Hd = H.toarray()
    left = w.gaussian_unit(p.H.m, 77, w.STREAM_LEFT, count=2)
    rf = oc.shifted_cocg(H, p.b, p.z, left=left, tol=p.tol, full=True)
    rp = oc.shifted_cocg(H, p.b, p.z, left=left, tol=p.tol, full=False)
    assert rf.status == oc.STATUS_OK and rp.status == oc.STATUS_OK
    xd = dense.dense_solutions(Hd, p.b, p.z)
    dist = dense.spectrum_distance(Hd, p.z)
    err = np.linalg.norm(rf.x - xd, axis=1)
    assert np.all(err <= 2 * p.tol / dist)
    lg = dense.lehmann_green(Hd, p.b, p.z, left)
    bound = (2 * p.tol / dist)[:, None]
    assert np.all(np.abs(rf.proj - lg) <= bound)
    assert np.all(np.abs(rp.proj - lg) <= bound)
    # true residuals (Eq. 7) within a small multiple of the recursive estimate
    tr = oc.true_residuals(H, p.b, p.z, rf.x)
    assert np.all(tr <= 10 * p.tol)


def test_lehmann_equals_dense_solve():
    Hd, b = _random_symmetric(25, 5)
    left = np.random.default_rng(1).standard_normal((2, 25))
    xd = dense.dense_solutions(Hd, b, Z5)
    lg = dense.lehmann_green(Hd, b, Z5, left)
    np.testing.assert_allclose(lg, xd @ np.vstack([b, left]).T, rtol=1e-12, atol=1e-13)
    # solutions satisfy Eq. 4
    for k, zk in enumerate(Z5):
        assert np.linalg.norm((zk * np.eye(25) - Hd) @ xd[k] - b) < 1e-12


def test_sum_rule():
    """-(1/pi) int Im b^T G(w + i delta) b dw = ||b||^2, on w = s tan(theta)."""
    H = w.anderson_3d(4, 2.0, seed=6).to_scipy()
    b = w.gaussian_unit(H.shape[0], 6)
    Nq, s, delta = 1024, 8.0, 0.2
    theta = -np.pi / 2 + (np.arange(Nq) + 0.5) * np.pi / Nq
    z = s * np.tan(theta) + 1j * delta
    r = oc.shifted_cocg(H, b, z, tol=1e-13, full=False)
    assert r.status == oc.STATUS_OK
    integrand = -np.imag(r.proj[:, 0]) / np.pi * s / np.cos(theta) ** 2
    total = integrand.sum() * np.pi / Nq
    assert abs(total - 1.0) < 1e-8


def test_large_z_moments():
    """b^T G(z) b = |b|^2/z + b^T H b/z^2 + b^T H^2 b/z^3 + O(|z|^-4)."""
    H = w.anderson_3d(5, 2.0, seed=8).to_scipy()
    b = w.gaussian_unit(H.shape[0], 8)
    z = np.array([1e3j, -1e3j, 1e3 + 1e3j, -2e3 + 5e2j])
    r = oc.shifted_cocg(H, b, z, tol=1e-15, full=False)
    Hb = H @ b
    m1, m2, m3 = b @ Hb, Hb @ Hb, Hb @ (H @ Hb)
    approx = 1 / z + m1 / z ** 2 + m2 / z ** 3
    assert np.all(np.abs(r.proj[:, 0] - approx) <= 2 * abs(m3) / np.abs(z) ** 4 + 1e-16)


def test_polarization_identity():
    """G_ab = (G_cc - G_aa - G_bb)/2 with c = a + b (real H, real a and b)."""
    H = w.anderson_3d(5, 4.0, seed=10).to_scipy()
    m = H.shape[0]
    a = w.gaussian_unit(m, 10, w.STREAM_LEFT)
    b = w.gaussian_unit(m, 10)
    z = w.shiftk_grid(-8, 8, 16, 0.1)
    tol = 1e-13
    g_ab = oc.shifted_cocg(H, b, z, left=a[None, :], tol=tol, full=False).proj[:, 1]
    g_aa = oc.shifted_cocg(H, a, z, tol=tol, full=False).proj[:, 0]
    g_bb = oc.shifted_cocg(H, b, z, tol=tol, full=False).proj[:, 0]
    c = a + b
    g_cc = oc.shifted_cocg(H, c, z, tol=tol, full=False).proj[:, 0]
    np.testing.assert_allclose(g_ab, (g_cc - g_aa - g_bb) / 2, atol=1e-9)


def test_seed_switching_neutral():
    """Seed switching changes only the rounding: early iterates agree to roundoff,
    converged solutions agree within the convergence bound."""
    p = w.anderson_small(L=5, K=16, delta=0.3, tol=1e-10)
    H = p.H.to_scipy()
    on = oc.shifted_cocg(H, p.b, p.z, tol=0.0, maxiter=15, full=True, seed_switch=True)
    off = oc.shifted_cocg(H, p.b, p.z, tol=0.0, maxiter=15, full=True, seed_switch=False)
    assert on.n_seed_switch > 0 and off.n_seed_switch == 0
    np.testing.assert_allclose(on.x, off.x, atol=1e-12)
    on = oc.shifted_cocg(H, p.b, p.z, tol=p.tol, full=True, seed_switch=True)
    off = oc.shifted_cocg(H, p.b, p.z, tol=p.tol, full=True, seed_switch=False)
    dist = dense.spectrum_distance(H.toarray(), p.z)
    assert np.all(np.linalg.norm(on.x - off.x, axis=1) <= 4 * p.tol / dist)


def test_real_shift_gives_real_solution():
    p = w.anderson_small(L=5, K=4)
    z = np.array([9.5 + 0j, -9.5 + 0j, 20.0 + 0j])
    r = oc.shifted_cocg(p.H.to_scipy(), p.b, z, tol=1e-12, full=True)
    assert r.status == oc.STATUS_OK
    assert np.abs(r.x.imag).max() < 1e-13


def test_degenerate_zero_matrix_and_eigenvector():
    M = 17
    b = w.gaussian_unit(M, 3)
    z = np.array([1 + 1j, -2 + 0.5j, 0.5j])
    r = oc.shifted_cocg(np.zeros((M, M)), b, z, tol=1e-14, full=True)
    assert r.iters == 1 and r.status == oc.STATUS_OK
    np.testing.assert_allclose(r.x, b[None, :] / z[:, None], rtol=1e-15)
    # b an eigenvector of H with eigenvalue 2: x = b / (z - 2) after one step
    Hd = 2.0 * np.eye(M)
    r = oc.shifted_cocg(Hd, b, z, tol=1e-14, full=True)
    assert r.iters == 1
    np.testing.assert_allclose(r.x, b[None, :] / (z[:, None] - 2.0), rtol=1e-14)


def test_diagonal_matrix_exact_in_distinct_eigenvalues():
    vals = np.array([-1.0, 0.5, 2.0, 3.5])
    d = np.repeat(vals, 5)
    b = w.gaussian_unit(d.size, 12)
    z = np.array([0.2 + 0.3j, 3 + 0.1j, -4 + 2j])
    r = oc.shifted_cocg(np.diag(d), b, z, tol=1e-13, full=True)
    assert r.iters <= vals.size + 1
    np.testing.assert_allclose(r.x, b[None, :] / (z[:, None] - d[None, :]), rtol=1e-12, atol=1e-14)


def test_maxiter_reports_not_converged():
    p = w.anderson_small(L=5, K=8)
    r = oc.shifted_cocg(p.H.to_scipy(), p.b, p.z, tol=1e-12, maxiter=5, full=False)
    assert r.status == oc.STATUS_NOT_CONVERGED and r.iters == 5
    assert np.all(r.conv_iter == -1)
    assert r.hist.shape == (5, 8)


def _krylov_basis(Hd, b, n):
    """Orthonormal basis of K_n(H, b) by Gram-Schmidt, twice per vector (stable
    where the power basis of _galerkin is not)."""
    M = b.size
    Q = np.zeros((M, n))
    v = b / np.linalg.norm(b)
    for i in range(n):
        Q[:, i] = v
        if i + 1 == n:
            break
        u = Hd @ v
        for _ in range(2):
            u -= Q[:, :i + 1] @ (Q[:, :i + 1].T @ u)
        v = u / np.linalg.norm(u)
    return Q


@pytest.mark.parametrize("switch", [True, False])
def test_freeze_rule_against_galerkin_residuals(switch):
    """Each shift is frozen at the first n whose Galerkin iterate has true
    residual <= tol ||b|| (here 12 to 21 iterations, every crossing at least 8%
    away from tol on both sides), keeps that iterate as x, and reports that
    residual in final_res."""
    Hd, b = _random_symmetric(30, 4)
    z = np.array([0.5 + 3j, -2 + 2.5j, 3 + 4j, 1 + 6j, -4 + 3.5j, 6 + 5j])
    tol = 1e-4
    r = oc.shifted_cocg(Hd, b, z, tol=tol, maxiter=30, full=True, seed_switch=switch)
    assert r.status == oc.STATUS_OK
    Q = _krylov_basis(Hd, b, 30)
    for k, zk in enumerate(z):
        A = zk * np.eye(b.size) - Hd
        xs, ts = [], []
        for n in range(1, 31):
            Qn = Q[:, :n]
            x = Qn @ np.linalg.solve(Qn.T @ A @ Qn, Qn.T @ b)
            xs.append(x)
            ts.append(np.linalg.norm(b - A @ x))
        ts = np.array(ts)
        c = int(np.argmax(ts <= tol)) + 1
        assert ts[c - 1] <= 0.92 * tol and (c == 1 or ts[c - 2] >= 1.05 * tol)
        assert r.conv_iter[k] == c, (k, r.conv_iter[k], c)
        assert np.linalg.norm(r.x[k] - xs[c - 1]) <= 1e-9 * np.linalg.norm(xs[c - 1])
        assert abs(r.final_res[k] - ts[c - 1]) <= 1e-9 * ts[c - 1]
