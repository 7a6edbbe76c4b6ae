"""GPU: reverse communication (kw_rci_init / kw_rci_update / kw_rci_get_residual /
kw_rci_finalize; the *_init, *_update, *_getresidual, *_finalize flow of
Sec. 3.1 (iii) and Algorithm 1).

The caller makes every product.  Driven by the same PyTorch product as a
kw_set_matvec solve, the reverse-communication solve runs the same kernels on
the same data and must give the same bits, in all three forms and for BiCG
(two products per iteration); the residuals it reports decrease to the
tolerance; it matches the oracle on the Anderson model.
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


def _stencil(L, eps):
    e = torch.as_tensor(eps, device="cuda")

    def fn(r, q):
        v = r.view(L, L, L)
        nb = sum(torch.roll(v, s, d) for d in range(3) for s in (1, -1))
        q.copy_((e.to(r.dtype).view(L, L, L) * v - nb).reshape(-1))
    return fn


def _drive(s, b, z, left, fn, fn_adj=None, full=False, cap=100000):
    r, q, rt, qt = s.rci_init(b, z, left=left, full=full)
    res_hist = []
    for _ in range(cap):
        fn(r, q)
        if rt is not None:
            fn_adj(rt, qt)
        done, (r, q, rt, qt) = s.rci_update()
        res_hist.append(s.rci_residual().max())
        if done:
            break
    return s.rci_finalize(check=False), res_hist


@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
def test_rci_equals_callback_solve(prec, full):
    L = 8
    H = w.anderson_3d(L, 2.0, seed=2)
    eps = H.to_scipy().diagonal().copy()
    b = w.gaussian_unit(H.m, 3)
    left = np.stack([w.gaussian_unit(H.m, 4 + i) for i in range(2)])
    z = w.shiftk_grid(-8, 8, 24, 0.05)
    tol = 1e-10 if prec != "c32" else 1e-7
    cb = kw.Solver(prec, tol=tol, maxiter=4000)
    cb.set_matvec(_stencil(L, eps), H.m)
    g = cb.solve(b, z, left=left, full=full, check=False)
    s = kw.Solver(prec, tol=tol, maxiter=4000)
    r, hist = _drive(s, b, z, left, _stencil(L, eps), full=full)
    assert (r.iters, r.status, r.n_seed_switch) == (g.iters, g.status, g.n_seed_switch)
    np.testing.assert_array_equal(r.proj, g.proj)
    if full:
        np.testing.assert_array_equal(r.x.cpu().numpy(), g.x.cpu().numpy())
    if prec != "c32":
        assert hist[-1] <= tol and r.status == "KW_OK"
        ro = oc.shifted_cocg(H.to_scipy(), b, z, left=left, tol=tol, full=False)
        ev = np.linalg.eigvalsh(H.to_scipy().toarray())
        dist = np.array([np.abs(zk - ev).min() for zk in z])
        scale = np.abs(ro.proj).max(axis=0)
        norms = np.linalg.norm(np.vstack([b, left]), axis=1)
        assert np.all(np.abs(r.proj - ro.proj) <= 1e-10 * scale[None, :] + 2 * tol * norms[None, :] / dist[:, None])


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_rci_bicg_equals_callback_bicg(prec):
    rng = np.random.default_rng(1)
    m = 100
    A = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    At = torch.as_tensor(A, device="cuda")
    Ah = torch.as_tensor(A.conj().T.copy(), device="cuda")
    fwd = lambda r, q: q.copy_(At.to(r.dtype) @ r)
    adj = lambda r, q: q.copy_(Ah.to(r.dtype) @ r)
    b = w.gaussian_unit(m, 3)
    z = np.array([2.5 + 0.3j, -2.2 + 0.5j, 0.3 + 2.0j, 3.0 - 1.0j])
    cb = kw.Solver(prec, tol=1e-10, maxiter=2000, method="bicg")
    cb.set_matvec(fwd, m, fn_adj=adj)
    g = cb.solve(b, z, full=True)
    s = kw.Solver(prec, tol=1e-10, maxiter=2000, method="bicg")
    r, _ = _drive(s, b, z, None, fwd, fn_adj=adj, full=True)
    assert (r.iters, r.status) == (g.iters, g.status) == (r.iters, "KW_OK")
    np.testing.assert_array_equal(r.proj, g.proj)
    np.testing.assert_array_equal(r.x.cpu().numpy(), g.x.cpu().numpy())


def test_rci_errors_and_state():
    s = kw.Solver("f64")
    assert s._lib.kw_rci_update(s._ctx, None, None) == kw.KW_ERR_ARG
    import ctypes as C
    d = C.c_int()
    io = kw.kw_rci_io()
    assert s._lib.kw_rci_update(s._ctx, C.byref(d), C.byref(io)) == kw.KW_ERR_ARG   # no kw_rci_init
