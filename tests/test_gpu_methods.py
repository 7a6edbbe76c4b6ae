"""GPU: the solvers of Table 1 besides COCG (kw_set_method; Appendix B).

* BiCG with the default shadow start (b, real) on a real symmetric H is COCG
  in exact arithmetic (r~_n = conj(r_n)); the GPU BiCG agrees with the oracle
  BiCG and with the GPU COCG within the parity bound, in all three forms.
* CG with real shifts on both sides of the spectrum agrees with the oracle CG
  (full x, element by element within the parity bound).
* A Hermitian complex H (callback, CG, real shifts) and a non-Hermitian complex
  H (callback with its adjoint, BiCG) against the dense definition, and BiCG
  iterates against the oracle BiCG after a fixed number of steps.
* Batched BiCG equals the individual BiCG solves; argument errors.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import shifted_bicg as ob
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


def _anderson(L=8, seed=3):
    H = w.anderson_3d(L, 2.0, seed=seed)
    b = w.gaussian_unit(H.m, seed + 1)
    left = np.stack([w.gaussian_unit(H.m, seed + 2 + i) for i in range(2)])
    return H, b, left


def _bound(Hd, b, left, z, tol, scale):
    ev = np.linalg.eigvalsh(Hd)
    dist = np.array([np.abs(zk - ev).min() for zk in z])
    norms = np.linalg.norm(np.vstack([b, left]), axis=1)
    return 1e-10 * scale[None, :] + 2 * tol * norms[None, :] / dist[:, None]


@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
def test_bicg_on_real_symmetric_matches_oracle_and_cocg(prec):
    H, b, left = _anderson()
    z = w.shiftk_grid(-8, 8, 32, 0.05)
    tol = 1e-10 if prec != "c32" else 1e-8
    s = kw.Solver(prec, tol=tol, maxiter=20000, method="bicg")
    s.set_csr(H.rowptr, H.col, H.val)
    r = s.solve(b, z, left=left, check=prec != "c32")
    ro = ob.shifted_bicg(H.to_scipy(), b, z, left=left, tol=tol, full=False, method="bicg")
    c = kw.Solver(prec, tol=tol, maxiter=20000)
    c.set_csr(H.rowptr, H.col, H.val)
    rc = c.solve(b, z, left=left, check=prec != "c32")
    scale = np.abs(ro.proj).max(axis=0)
    if prec == "c32":
        assert np.abs(r.proj - ro.proj).max() <= 1e-5 * scale.max()
        return
    assert r.status == "KW_OK" and abs(r.iters - ro.iters) <= 0.05 * ro.iters + 2
    bound = _bound(H.to_scipy().toarray(), b, left, z, tol, scale)
    assert np.all(np.abs(r.proj - ro.proj) <= bound)
    assert np.all(np.abs(r.proj - rc.proj) <= bound)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_cg_real_shifts_matches_oracle(prec):
    H, b, left = _anderson(L=6, seed=5)
    Hs = H.to_scipy()
    ev = np.linalg.eigvalsh(Hs.toarray())
    z = np.concatenate([np.linspace(ev[0] - 3, ev[0] - 0.3, 5), np.linspace(ev[-1] + 0.3, ev[-1] + 3, 5)])
    s = kw.Solver(prec, tol=1e-11, maxiter=5000, method="cg")
    s.set_csr(H.rowptr, H.col, H.val)
    r = s.solve(b, z, left=left, full=True)
    ro = ob.shifted_bicg(Hs, b, z.astype(np.complex128), left=left, tol=1e-11, full=True, method="cg")
    assert r.status == "KW_OK" and abs(r.iters - ro.iters) <= 2
    x = r.x.cpu().numpy()
    dist = np.array([np.abs(zk - ev).min() for zk in z])
    err = np.linalg.norm(x - ro.x, axis=1)
    assert np.all(err <= 1e-10 * np.linalg.norm(ro.x, axis=1) + 2e-11 / dist)


def _torch_dense_op(A, dtype=torch.complex128):
    At = torch.as_tensor(A, device="cuda", dtype=dtype)

    def fn(r, q):
        q.copy_(At.to(r.dtype) @ r)
    return fn


def test_cg_hermitian_callback_against_dense():
    rng = np.random.default_rng(2)
    m = 160
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    H = (A + A.conj().T) / (2 * np.sqrt(m))
    b = w.gaussian_unit(m, 7)
    ev = np.linalg.eigvalsh(H)
    z = np.concatenate([np.linspace(ev[0] - 2, ev[0] - 0.2, 4), np.linspace(ev[-1] + 0.2, ev[-1] + 2, 4)])
    s = kw.Solver("f64", tol=1e-11, maxiter=2000, method="cg")
    s.set_matvec(_torch_dense_op(H), m)
    r = s.solve(b, z, full=True)
    assert r.status == "KW_OK"
    x = r.x.cpu().numpy()
    _, fr = s.shift_status(z.size)
    for k, zk in enumerate(z):
        Ak = zk * np.eye(m) - H
        xk = np.linalg.solve(Ak, b)
        smin = np.linalg.svd(Ak, compute_uv=False)[-1]
        assert np.linalg.norm(x[k] - xk) <= 2 * max(fr[k], 1e-13) / smin + 1e-12


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_bicg_nonhermitian_callback(prec):
    rng = np.random.default_rng(1)
    m = 120
    A = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    b = w.gaussian_unit(m, 3)
    z = np.array([2.5 + 0.3j, -2.2 + 0.5j, 0.3 + 2.0j, 3.0 - 1.0j, 0.5 + 1.5j])
    s = kw.Solver(prec, tol=1e-10, maxiter=3000, method="bicg")
    s.set_matvec(_torch_dense_op(A), m, fn_adj=_torch_dense_op(A.conj().T))
    r = s.solve(b, z, full=True)
    assert r.status == "KW_OK"
    x = r.x.cpu().numpy()
    _, fr = s.shift_status(z.size)
    for k, zk in enumerate(z):
        Ak = zk * np.eye(m) - A
        xk = np.linalg.solve(Ak, b)
        smin = np.linalg.svd(Ak, compute_uv=False)[-1]
        assert np.linalg.norm(x[k] - xk) <= 2 * max(fr[k], 1e-13) / smin + 1e-12
    # fixed number of steps: the GPU iterates are the oracle's
    n = 15
    s2 = kw.Solver(prec, tol=0.0, maxiter=n, method="bicg")
    s2.set_matvec(_torch_dense_op(A), m, fn_adj=_torch_dense_op(A.conj().T))
    g = s2.solve(b, z, full=True, check=False)
    ro = ob.shifted_bicg(A, b, z, tol=0.0, maxiter=n, full=True, method="bicg")
    assert g.iters == n
    gx = g.x.cpu().numpy()
    assert np.abs(gx - ro.x).max() <= (1e-11 if prec == "f64" else 1e-10) * np.abs(ro.x).max()


def test_batched_bicg_equals_individual():
    batch = []
    for i in range(3):
        H, b, left = _anderson(L=5 + i, seed=10 + i)
        batch.append({"H": H, "b": b, "z": w.shiftk_grid(-8, 8, 12 + 4 * i, 0.05), "tol": 1e-9,
                      "full": i != 1})
    res = kw.Solver("f64", maxiter=5000, method="bicg").solve_batched(batch)
    for d, r in zip(batch, res):
        one = kw.Solver("f64", maxiter=5000, tol=d["tol"], method="bicg")
        one.set_csr(d["H"].rowptr, d["H"].col, d["H"].val)
        g = one.solve(d["b"], d["z"], full=d["full"])
        assert (r.iters, r.status) == (g.iters, g.status)
        np.testing.assert_array_equal(r.proj, g.proj)


def test_method_arguments():
    H, b, _ = _anderson(L=4)
    s = kw.Solver("f64", method="cg")
    s.set_csr(H.rowptr, H.col, H.val)
    with pytest.raises(kw.KomegaError) as ei:
        s.solve(b, [0.1 + 0.1j])                     # CG needs real shifts
    assert ei.value.status == kw.KW_ERR_ARG
    assert s._lib.kw_set_method(s._ctx, 7, None) == kw.KW_ERR_ARG
    with pytest.raises(kw.KomegaError):
        s.set_method("cg", btilde=b)                 # a shadow start is for BiCG only
