"""GPU: continuing a stopped solve (kw_resume; the restart mode of Sec. 3.3).

A solve capped at n1 iterations and resumed to convergence must give what one
solve with the larger cap gives: bit for bit in the FP64 and FP32 forms and in
the pair form's projected mode (the same kernels run on the same state); the
pair form's x went through kw_c128 and back, which keeps its value.  Also with
BiCG, several resumes in a row, the Krylov log continuing, and the cases that
must be refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()


def _problem():
    H = w.anderson_3d(9, 2.0, seed=6)
    b = w.gaussian_unit(H.m, 7)
    left = np.stack([w.gaussian_unit(H.m, 8 + i) for i in range(2)])
    z = w.shiftk_grid(-8, 8, 40, 0.05)
    return H, b, left, z


def _solver(H, prec, maxiter, method="cocg"):
    s = kw.Solver(prec, tol=1e-10, maxiter=maxiter, method=method)
    s.set_csr(H.rowptr, H.col, H.val)
    return s


@pytest.mark.parametrize("method", ["cocg", "bicg"])
@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
def test_resume_equals_single_solve(prec, full, method):
    H, b, left, z = _problem()
    one = _solver(H, prec, 20000, method).solve(b, z, left=left, full=full, check=False)
    s = _solver(H, prec, 137, method)
    a = s.solve(b, z, left=left, full=full, check=False)
    assert a.status == "KW_NOT_CONVERGED" and a.iters == 137
    r = s.resume(20000 - 137, check=False)
    assert (r.iters, r.status, r.n_seed_switch, r.updates) == (one.iters, one.status, one.n_seed_switch, one.updates)
    np.testing.assert_array_equal(r.proj, one.proj)
    if full:
        xa, xb = r.x.cpu().numpy(), one.x.cpu().numpy()
        if prec == "df64":
            assert np.abs(xa - xb).max() <= 1e-14 * np.abs(xb).max()
        else:
            np.testing.assert_array_equal(xa, xb)


def test_repeated_resumes_and_log():
    H, b, left, z = _problem()
    one = _solver(H, "f64", 20000)
    one.set_krylov_log(100000)
    ro = one.solve(b, z, left=left)
    s = _solver(H, "f64", 50)
    s.set_krylov_log(100000)
    r = s.solve(b, z, left=left, check=False)
    while r.status == "KW_NOT_CONVERGED":
        r = s.resume(77, check=False)
    assert r.iters == ro.iters
    np.testing.assert_array_equal(r.proj, ro.proj)
    np.testing.assert_array_equal(s.krylov_log().rows, one.krylov_log().rows)


def test_resume_refused():
    H, b, left, z = _problem()
    s = _solver(H, "f64", 20000)
    with pytest.raises(kw.KomegaError):
        s.resume(10)                                 # nothing solved yet
    s.solve(b, z, left=left)
    with pytest.raises(kw.KomegaError):
        s.resume(10)                                 # converged: nothing to continue
    s2 = _solver(H, "f64", 30)
    s2.solve(b, z, left=left, check=False)
    s2.set_csr(H.rowptr, H.col, H.val)               # operator set again
    with pytest.raises(kw.KomegaError):
        s2.resume(10)
