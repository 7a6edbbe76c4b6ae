"""GPU: the row-group form of the three-term update (kw_set_seed_update).

In the FP32-pair form, each 256-element tile forms r_{n+1} (Eq. 16) one element
per thread, then four thread groups form every fourth projection row
w_l = a_l^T r_{n+1} (Eq. 26) from shared memory.  Only the summation order of
the dots differs from the one-element-per-thread kernel, so after a few
iterations both agree to pair rounding (1e-12 of the largest projection);
converged solves agree with the oracle within the convergence bound; the
default picks the row-group form above nine projection rows and equals that
choice bit for bit; CG (real shifts) uses it too; m below one tile, one whole
tile and ragged tiles, 1 to 31 left vectors.
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


def _ring(m, seed=3):
    rng = np.random.default_rng(seed)
    i = np.arange(m)
    rows = np.concatenate([i, i, i])
    cols = np.concatenate([i, (i + 1) % m, (i - 1) % m])
    vals = np.concatenate([rng.uniform(-1.0, 1.0, m), -np.ones(m), -np.ones(m)])
    return w._csr_from_coo(m, rows, cols, vals)


def _run(m, nleft, mode, full=False, maxiter=8, method="cocg", z=None, tol=1e-9):
    H = _ring(m)
    b = w.gaussian_unit(m, 21)
    left = np.stack([w.gaussian_unit(m, 22 + i) for i in range(nleft)]) if nleft else None
    z = w.shiftk_grid(-3, 3, 24, 0.04) if z is None else z
    s = kw.Solver("df64", tol=tol, maxiter=maxiter, method=method)
    s.set_seed_update(mode)
    s.set_csr(H.rowptr, H.col, H.val)
    r = s.solve(b, z, left=left, full=full, check=False)
    return r, (H, b, left, z)


@pytest.mark.parametrize("m,nleft,full", [(200, 16, False), (256, 10, False), (4113, 16, False), (4113, 31, False),
                                          (20001, 12, False), (3072, 1, False), (4113, 4, True)])
def test_row_groups_agree_with_one_element_per_thread(m, nleft, full):
    a, _ = _run(m, nleft, 1, full)
    b, _ = _run(m, nleft, 0, full)
    assert (a.iters, a.status) == (b.iters, b.status) == (8, "KW_NOT_CONVERGED")
    assert np.abs(a.proj - b.proj).max() <= 1e-12 * np.abs(b.proj).max()
    if full:
        xa, xb = a.x.cpu().numpy(), b.x.cpu().numpy()
        assert np.abs(xa - xb).max() <= 1e-12 * np.abs(xb).max()


def test_row_groups_converged_against_oracle():
    r, (H, b, left, z) = _run(4113, 16, 1, maxiter=3000)
    assert r.status == "KW_OK"
    ref = oc.shifted_cocg(H.to_scipy(), b, z, left=left, tol=1e-9, full=False)
    err = np.abs(r.proj - ref.proj).max(axis=1) * np.abs(z.imag)
    assert err.max() < 4e-9, err.max()


@pytest.mark.parametrize("nleft,rg", [(16, True), (9, True), (8, False), (2, False)])
def test_default_uses_row_groups_above_nine_rows(nleft, rg):
    d, _ = _run(4113, nleft, -1)
    f, _ = _run(4113, nleft, 1 if rg else 0)
    np.testing.assert_array_equal(d.proj, f.proj)


def test_row_groups_with_cg_real_shifts():
    z = np.linspace(-6.0, -3.5, 16).astype(np.complex128)     # below the ring's spectrum (>= -3)
    a, _ = _run(4113, 12, 1, maxiter=400, method="cg", z=z, tol=1e-10)
    b, (H, bb, left, _) = _run(4113, 12, 0, maxiter=400, method="cg", z=z, tol=1e-10)
    assert a.status == b.status == "KW_OK"
    assert abs(a.iters - b.iters) <= 1
    ref = oc.shifted_cocg(H.to_scipy(), bb, z, left=left, tol=1e-10, full=False)
    assert np.abs(a.proj - ref.proj).max() <= 1e-8 * np.abs(ref.proj).max()


def test_seed_update_argument():
    s = kw.Solver("df64")
    assert s._lib.kw_set_seed_update(s._ctx, 2) == kw.KW_ERR_ARG
    assert s._lib.kw_set_seed_update(s._ctx, -2) == kw.KW_ERR_ARG


def test_row_groups_bounded_wait_reports_timeout_and_context_recovers():
    """The row-group kernel stages the projection rows with TMA bulk copies on
    bounded mbarrier waits: armed for 16 bytes more than its copies bring
    (kw_set_bulk_copy(2)), the wait runs out, the solve ends with
    KW_ERR_TIMEOUT, and the context then solves correctly."""
    m, nleft = 4113, 12
    H = _ring(m)
    b = w.gaussian_unit(m, 21)
    left = np.stack([w.gaussian_unit(m, 22 + i) for i in range(nleft)])
    z = w.shiftk_grid(-3, 3, 8, 0.04)
    s = kw.Solver("df64", tol=1e-9, maxiter=3000)
    s.set_seed_update(1)
    s.set_csr(H.rowptr, H.col, H.val)
    good = s.solve(b, z, left=left)
    s.set_bulk_copy(2)
    bad = s.solve(b, z, left=left, check=False)
    assert bad.status == "KW_ERR_TIMEOUT"
    assert bad.iters <= 8
    s.set_bulk_copy(-1)
    again = s.solve(b, z, left=left)
    assert again.iters == good.iters
    np.testing.assert_array_equal(again.proj, good.proj)
