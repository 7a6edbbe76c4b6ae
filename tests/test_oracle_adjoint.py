"""CPU pins for the oracle gradient of the spectrum (oracle/adjoint.py).

* Dense: dA_k/dtheta_m from the explicit inverse, -(1/pi) Im b^T G H_m G b.
* Central differences of the oracle's own spectrum (forward solves only).
* A step along -grad lowers the loss.
"""
import numpy as np

from oracle import adjoint as oa
from paper_2001_08707_gb300 import workloads as w


def _model(N=8, seed=3):
    j = w.j1j2_chain(N, 1.0, 0.4, 0.2, seed=seed)
    terms = [t.to_scipy() for t in j.terms]
    b = w.gaussian_unit(j.terms[0].m, seed)
    z = w.shiftk_grid(-3.0, 2.0, 12, 0.2)
    return j, terms, b, z


def test_gradient_matches_dense_inverse():
    j, terms, b, z = _model()
    _, _, _, dA = oa.spectrum_and_gradient(terms, j.theta, b, z, np.zeros(z.size), tol=1e-13)
    H = oa.assemble(terms, j.theta).toarray()
    M = H.shape[0]
    for k, zk in enumerate(z):
        G = np.linalg.inv(zk * np.eye(M) - H)
        for m, Hm in enumerate(terms):
            ref = -np.imag(b @ G @ Hm.toarray() @ G @ b) / np.pi
            assert abs(dA[k, m] - ref) <= 1e-9 * (1 + abs(ref))


def test_gradient_matches_central_differences():
    j, terms, b, z = _model(N=10, seed=5)
    rng = np.random.default_rng(0)
    target = oa.spectrum(terms, j.theta + rng.normal(0, 0.05, j.theta.size), b, z, tol=1e-13)[0]
    A, loss, grad, _ = oa.spectrum_and_gradient(terms, j.theta, b, z, target, tol=1e-13)
    h = 1e-5
    for m in range(j.theta.size):
        e = np.zeros_like(j.theta)
        e[m] = h
        Ap = oa.spectrum(terms, j.theta + e, b, z, tol=1e-13)[0]
        Am = oa.spectrum(terms, j.theta - e, b, z, tol=1e-13)[0]
        fd = (0.5 * np.sum((Ap - target) ** 2) - 0.5 * np.sum((Am - target) ** 2)) / (2 * h)
        assert abs(fd - grad[m]) <= 1e-6 * (abs(grad[m]) + 1e-3), (m, fd, grad[m])


def test_descent_direction_lowers_loss():
    j, terms, b, z = _model()
    target = oa.spectrum(terms, j.theta * 1.02, b, z, tol=1e-13)[0]
    _, loss, grad, _ = oa.spectrum_and_gradient(terms, j.theta, b, z, target, tol=1e-13)
    _, loss2, _, _ = oa.spectrum_and_gradient(terms, j.theta - 1e-3 * grad / np.linalg.norm(grad), b, z, target,
                                              tol=1e-13)
    assert loss2 < loss


def test_assemble_matches_the_generators():
    """oracle.adjoint.assemble against two builds that share none of its code:
    the generator's own COO assembly of H(theta), and, for theta = (1, 0, 0, ...),
    the nearest-neighbour Heisenberg chain built bond by bond (Eq. 41)."""
    j = w.j1j2_chain(8, 1.0, 0.4, 0.2, seed=3)
    terms = [t.to_scipy() for t in j.terms]
    A = oa.assemble(terms, j.theta).toarray()
    B = j.assemble().to_scipy().toarray()
    np.testing.assert_allclose(A, B, rtol=0, atol=1e-15)
    th = np.zeros_like(j.theta)
    th[0] = 1.0
    C = oa.assemble(terms, th).toarray()
    np.testing.assert_allclose(C, w.heisenberg_chain(8).to_scipy().toarray(), rtol=0, atol=1e-15)
    # every term enters: dropping the last field term changes the matrix
    assert np.abs(oa.assemble(terms[:-1], j.theta[:-1]).toarray() - A).max() > 1e-3


def test_green_gradient_a_ne_b_matches_dense_inverse_and_is_symmetric():
    """dG_ab/dtheta_m = a^T G H_m G b with G the explicit inverse, for a left vector
    a different from b; and swapping a and b gives the same derivative (G and H_m
    symmetric), which a transposed operand or a y/x mix-up would break."""
    j, terms, b, z = _model(N=8, seed=4)
    a = w.gaussian_unit(j.terms[0].m, 9, w.STREAM_LEFT)
    G, dG = oa.green_and_gradient(terms, j.theta, a, b, z, tol=1e-13)
    H = oa.assemble(terms, j.theta).toarray()
    M = H.shape[0]
    for k, zk in enumerate(z):
        Gi = np.linalg.inv(zk * np.eye(M) - H)
        assert abs(G[k] - a @ Gi @ b) <= 1e-10 * (1 + abs(G[k]))
        for m, Hm in enumerate(terms):
            ref = a @ Gi @ Hm.toarray() @ Gi @ b
            assert abs(dG[k, m] - ref) <= 1e-9 * (1 + abs(ref))
    G2, dG2 = oa.green_and_gradient(terms, j.theta, b, a, z, tol=1e-13)
    np.testing.assert_allclose(G2, G, rtol=0, atol=1e-10 * np.abs(G).max())
    np.testing.assert_allclose(dG2, dG, rtol=0, atol=1e-9 * np.abs(dG).max())
    # a = b reduces to the spectrum gradient: dA/dtheta = -(1/pi) Im dG_bb/dtheta
    _, _, _, dA = oa.spectrum_and_gradient(terms, j.theta, b, z, np.zeros(z.size), tol=1e-13)
    _, dGbb = oa.green_and_gradient(terms, j.theta, b, b, z, tol=1e-13)
    np.testing.assert_allclose(-np.imag(dGbb) / np.pi, dA, rtol=0, atol=1e-10 * np.abs(dA).max())


def test_green_gradient_a_ne_b_central_differences():
    j, terms, b, z = _model(N=10, seed=6)
    a = w.gaussian_unit(j.terms[0].m, 11, w.STREAM_LEFT)
    _, dG = oa.green_and_gradient(terms, j.theta, a, b, z, tol=1e-13)
    h = 1e-5
    for m in (0, 1, 3):
        e = np.zeros_like(j.theta)
        e[m] = h
        Gp, _ = oa.green_and_gradient(terms, j.theta + e, a, b, z, tol=1e-13)
        Gm, _ = oa.green_and_gradient(terms, j.theta - e, a, b, z, tol=1e-13)
        fd = (Gp - Gm) / (2 * h)
        assert np.abs(fd - dG[:, m]).max() <= 1e-6 * np.abs(dG[:, m]).max()
