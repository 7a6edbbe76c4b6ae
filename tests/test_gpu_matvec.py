"""GPU: the operator given as a caller's matrix-vector callback (kw_set_matvec).

The callbacks here are matrix-free PyTorch operators (Sec. 3.1 (i): the
product is left to the application): the Anderson Hamiltonian as a 7-point
periodic stencil with torch.roll, and a complex symmetric variant (an
imaginary onsite potential).  Checks:

* one K1 step through the callback equals the CSR kernel's (1e-14 relative);
* converged solves through the callback agree with the oracle (the CSR matrix
  of the same Hamiltonian) within the parity bound, in all three forms;
* a complex symmetric H (allowed through the callback, COCG needs only
  A = zI - H complex symmetric) against the dense definition;
* a failing callback stops the solve with KW_ERR_CALLBACK and the context
  stays usable; kw_set_csr ends the callback.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()


def _anderson(L, seed):
    H = w.anderson_3d(L, 2.0, seed=seed)
    Hs = H.to_scipy()
    eps = Hs.diagonal().copy()
    return H, Hs, eps


class Stencil:
    """q = H r for the periodic Anderson model: eps_i r_i - sum of the 6 neighbours
    (hopping -1; site i = x + L(y + L z), so the reshape is [z, y, x])."""

    def __init__(self, L, eps, imag=None):
        self.L = L
        e = torch.as_tensor(eps, device="cuda")
        if imag is not None:
            e = torch.complex(e, torch.as_tensor(imag, device="cuda"))
        self.eps = e
        self.calls = 0

    def __call__(self, r, q):
        self.calls += 1
        L = self.L
        v = r.view(L, L, L)
        nb = sum(torch.roll(v, s, d) for d in range(3) for s in (1, -1))
        out = self.eps.to(r.dtype).view(L, L, L) * v - nb
        q.copy_(out.reshape(-1))


def test_one_step_matches_csr_kernel():
    L = 12
    H, _, eps = _anderson(L, 3)
    rng = np.random.default_rng(0)
    r = torch.as_tensor(rng.standard_normal(H.m) + 1j * rng.standard_normal(H.m), device="cuda")
    a = kw.Solver("f64")
    a.set_csr(H.rowptr, H.col, H.val)
    qa = torch.empty_like(r)
    ta = a.spmv_dot(0.3 + 0.7j, r, qa)
    b = kw.Solver("f64")
    op = Stencil(L, eps)
    b.set_matvec(op, H.m)
    qb = torch.empty_like(r)
    tb = b.spmv_dot(0.3 + 0.7j, r, qb)
    assert op.calls == 1
    assert (qa - qb).abs().max().item() <= 1e-14 * qa.abs().max().item()
    assert abs(ta - tb) <= 1e-13 * abs(ta)


@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
def test_converged_solve_through_callback_matches_oracle(prec):
    L = 10
    H, Hs, eps = _anderson(L, 1)
    b = w.gaussian_unit(H.m, 11)
    left = np.stack([w.gaussian_unit(H.m, 12 + i) for i in range(2)])
    z = w.shiftk_grid(-8, 8, 32, 0.05)
    tol = 1e-10 if prec != "c32" else 1e-8
    s = kw.Solver(prec, tol=tol, maxiter=20000)
    op = Stencil(L, eps)
    s.set_matvec(op, H.m)
    r = s.solve(b, z, left=left)
    ro = oc.shifted_cocg(Hs, b, z, left=left, tol=tol, full=False)
    assert op.calls >= r.iters
    scale = np.abs(ro.proj).max(axis=0)
    err = (np.abs(r.proj - ro.proj).max(axis=0) / scale).max()
    if prec == "c32":
        assert err <= 1e-5
    else:
        assert r.status == "KW_OK" and abs(r.iters - ro.iters) <= 0.05 * ro.iters
        ev = np.linalg.eigvalsh(Hs.toarray())
        dist = np.array([np.abs(zk - ev).min() for zk in z])
        bound = 1e-10 * scale[None, :] + 2 * tol * np.linalg.norm(np.vstack([b, left]), axis=1)[None, :] / dist[:, None]
        assert np.all(np.abs(r.proj - ro.proj) <= bound)


def test_complex_symmetric_operator_against_dense():
    L = 8
    H, Hs, eps = _anderson(L, 5)
    rng = np.random.default_rng(4)
    gamma = -0.3 * rng.random(H.m)                # absorbing onsite term: H = H_0 + i diag(gamma)
    b = w.gaussian_unit(H.m, 6)
    z = w.shiftk_grid(-8, 8, 24, 0.05)
    s = kw.Solver("f64", tol=1e-10, maxiter=20000)
    s.set_matvec(Stencil(L, eps, imag=gamma), H.m)
    r = s.solve(b, z, full=True)
    assert r.status == "KW_OK"
    Hd = Hs.toarray() + 1j * np.diag(gamma)
    X = np.stack([np.linalg.solve(zk * np.eye(H.m) - Hd, b) for zk in z])
    x = r.x.cpu().numpy()
    # residual of the GPU iterate against the dense operator, and the solution error it bounds
    res = np.array([np.linalg.norm(b - (zk * x[k] - Hd @ x[k])) for k, zk in enumerate(z)])
    assert np.all(res <= 10 * 1e-10)
    smin = np.array([np.linalg.svd(zk * np.eye(H.m) - Hd, compute_uv=False)[-1] for zk in z])
    assert np.all(np.linalg.norm(x - X, axis=1) <= 2 * res / smin + 1e-13)


def test_failing_callback_reports_and_context_recovers():
    L = 6
    H, Hs, eps = _anderson(L, 2)
    b = w.gaussian_unit(H.m, 3)
    z = w.shiftk_grid(-8, 8, 8, 0.1)
    s = kw.Solver("f64", tol=1e-10)

    def broken(r, q):
        raise ValueError("planted failure")

    s.set_matvec(broken, H.m)
    with pytest.raises(kw.KomegaError) as ei:
        s.solve(b, z)
    assert ei.value.status == kw.KW_ERR_CALLBACK and isinstance(ei.value.__cause__, ValueError)
    s.set_matvec(Stencil(L, eps), H.m)          # the same context works again
    ok = s.solve(b, z)
    s.set_csr(H.rowptr, H.col, H.val)           # and back to the CSR kernel
    ref = s.solve(b, z)
    assert ok.status == ref.status == "KW_OK"
    assert np.abs(ok.proj - ref.proj).max() <= 1e-9 * np.abs(ref.proj).max()


def test_set_matvec_arguments():
    s = kw.Solver("f64")
    with pytest.raises(kw.KomegaError):
        s.set_matvec(lambda r, q: None, 0)
