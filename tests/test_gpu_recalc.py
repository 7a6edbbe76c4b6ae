"""GPU parity for recalculation at new shifts (kw_set_krylov_log, kw_get_krylov_log, kw_recalc).

* The device log of a short FP64 run matches the oracle's log entry by entry
  (same algorithm, rounding order only: 1e-10 relative per column over 30
  iterations on the L=12 Anderson model, the regime where the plain parity
  tests hold 1e-11).
* kw_recalc on the oracle's own log (uploaded from the host) matches the
  oracle's replay of that log: same inputs, rounding only (1e-11).
* Recalculation from the device log at shifts that were not solved agrees
  with the dense definition within the residual bound, in all three precision
  forms, and with a direct GPU solve at those shifts.
* Replaying the solved shifts reproduces the solve; truncated logs and an
  empty log behave like a solve stopped at that iteration.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import recalc as orc
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


def _problem(L=10, seed=3, nleft=3, K=48, delta=0.05):
    H = w.anderson_3d(L, 2.0, seed=seed)
    b = w.gaussian_unit(H.m, seed + 2)
    left = np.stack([w.gaussian_unit(H.m, seed + 3 + i) for i in range(nleft)])
    z = w.shiftk_grid(-8, 8, K, delta)
    return H, b, left, z


def _solver(H, prec="f64", **opts):
    s = kw.Solver(prec, **opts)
    s.set_csr(H.rowptr, H.col, H.val)
    return s


def _oracle_rows(lg):
    """The oracle's KrylovLog in the C-ABI row layout (test-side conversion)."""
    fixed = np.stack([lg.zs, lg.alpha, lg.c, lg.beta, lg.nu.astype(np.complex128), lg.pj1, lg.pj0], axis=1)
    return np.ascontiguousarray(np.concatenate([fixed, lg.w], axis=1))


def _dense_bound(H, b, left, z, final_res, factor=2.0):
    Hd = H.to_scipy().toarray()
    M = b.size
    X = np.stack([np.linalg.solve(zk * np.eye(M) - Hd, b) for zk in z])
    ev = np.linalg.eigvalsh(Hd)
    dist = np.array([np.abs(zk - ev).min() for zk in z])
    P = np.vstack([b, left])
    norms = np.linalg.norm(P, axis=1)
    return X @ P.T, factor * final_res[:, None] * norms[None, :] / dist[:, None]


def test_device_log_matches_oracle_log():
    H, b, left, z = _problem(L=12, seed=5, K=16)
    n = 30
    s = _solver(H, "f64", tol=1e-10, maxiter=n)
    s.set_krylov_log(1000)
    s.solve(b, z, left=left)
    lg = s.krylov_log()
    ro = oc.shifted_cocg(H.to_scipy(), b, z, left=left, tol=1e-10, maxiter=n, full=False, log=True)
    ref = _oracle_rows(ro.log)
    assert lg.rows.shape == ref.shape and lg.n_run == n
    np.testing.assert_array_equal(lg.rows[:, 0], ref[:, 0])            # same seeds
    for col in range(1, kw.LOG_FIXED):
        scale = np.abs(ref[:, col]).max()
        assert np.abs(lg.rows[:, col] - ref[:, col]).max() <= 1e-10 * scale, col
    # P r_{n+1}: a dot product's rounding scales with ||a_l|| ||r_{n+1}|| (b^T r_{n+1} is 0 in
    # exact arithmetic, so the entry itself is rounding)
    norms = np.linalg.norm(np.vstack([b, left]), axis=1)
    scale = np.sqrt(ro.log.nu)[:, None] * norms[None, :]
    assert np.all(np.abs(lg.rows[:, kw.LOG_FIXED:] - ref[:, kw.LOG_FIXED:]) <= 1e-10 * scale)
    assert np.abs(lg.w0 - ro.log.w0).max() <= 1e-13
    assert abs(lg.thresh - ro.log.thresh) <= 1e-15 * ro.log.thresh


@pytest.mark.parametrize("nleft", [0, 3, 20])
def test_recalc_of_oracle_log_matches_oracle_replay(nleft):
    H, b, left, z = _problem(L=8, seed=7, nleft=max(nleft, 1))
    left = left[:nleft] if nleft else None
    ro = oc.shifted_cocg(H.to_scipy(), b, z, left=left, tol=1e-10, full=False, log=True)
    znew = np.concatenate([z + 0.17 + 0.03j, [3e2j, -0.4 + 2.0j]])
    ref = orc.recalc(ro.log, znew)
    log = kw.KrylovLog(_oracle_rows(ro.log), ro.log.w0, ro.log.thresh, ro.iters)
    s = _solver(H, "f64", tol=1e-10)
    got = s.recalc(znew, log=log)
    np.testing.assert_array_equal(got.conv_iter, ref.conv_iter)
    assert np.abs(got.proj - ref.proj).max() <= 1e-11 * np.abs(ref.proj).max()
    fin = np.isfinite(ref.final_res)
    assert np.all(np.abs(got.final_res[fin] - ref.final_res[fin]) <= 1e-11 * ref.final_res[fin])


@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
def test_recalc_from_device_log_matches_dense(prec):
    H, b, left, z = _problem(L=10, seed=3)
    tol = 1e-10 if prec != "c32" else 1e-8
    s = _solver(H, prec, tol=tol, maxiter=20000)
    s.set_krylov_log(20000)
    r = s.solve(b, z, left=left)
    znew = z + 0.17 + 0.15j                     # midpoints, further from the axis
    rc = s.recalc(znew)
    assert rc.iters == r.iters
    if prec != "c32":                           # the FP32-vector form may stall above tol
        assert r.status == "KW_OK" and rc.status == "KW_OK"
    ref, bound = _dense_bound(H, b, left, znew, rc.final_res)
    if prec == "c32":                           # FP32 vectors: checked on the spectrum error
        assert np.abs(rc.proj - ref).max() <= 1e-5 * np.abs(ref).max()
    else:
        assert np.all(np.abs(rc.proj - ref) <= bound + 1e-12)
    d = s.solve(b, znew, left=left)             # direct GPU solve at the new shifts
    scale = np.abs(d.proj).max()
    assert np.abs(rc.proj - d.proj).max() <= (1e-5 if prec == "c32" else 1e-8) * scale


def test_recalc_of_own_shifts_reproduces_solve():
    H, b, left, z = _problem(L=10, seed=9, K=64)
    s = _solver(H, "f64", tol=1e-10)
    s.set_krylov_log(100000)
    r = s.solve(b, z, left=left)
    ci, _ = s.shift_status(z.size)
    rc = s.recalc(z)
    np.testing.assert_array_equal(rc.conv_iter, ci)
    assert np.abs(rc.proj - r.proj).max() <= 1e-12 * np.abs(r.proj).max()


@pytest.mark.parametrize("cut", [0, 1, 9, 50])
def test_truncated_log_replays_stopped_solve(cut):
    H, b, left, z = _problem(L=8, seed=2, K=24)
    s = _solver(H, "f64", tol=1e-10)
    s.set_krylov_log(cut)
    r = s.solve(b, z, left=left)
    if cut == 0:                                # logging off: no log to read
        with pytest.raises(kw.KomegaError):
            s.krylov_log()
        return
    lg = s.krylov_log()
    assert lg.rows.shape[0] == cut and lg.n_run == r.iters > cut
    rc = s.recalc(z)
    stop = _solver(H, "f64", tol=1e-10, maxiter=cut)
    rs = stop.solve(b, z, left=left)
    ci, _ = stop.shift_status(z.size)
    assert rc.status == "KW_NOT_CONVERGED" and rc.iters == cut
    np.testing.assert_array_equal(rc.conv_iter, ci)
    assert np.abs(rc.proj - rs.proj).max() <= 1e-12 * np.abs(rs.proj).max()
    # the same rows uploaded from the host give the same answer
    rh = s.recalc(z, log=lg)
    np.testing.assert_array_equal(rh.proj, rc.proj)


def test_empty_host_log_and_single_shift():
    s = _solver(w.anderson_3d(4, 2.0, seed=1), "f64")
    log = kw.KrylovLog(np.zeros((0, kw.LOG_FIXED + 2), np.complex128), np.array([1.0, 0.5], np.complex128),
                       1e-10, 0)
    rc = s.recalc([0.3 + 0.1j], log=log)
    assert rc.status == "KW_NOT_CONVERGED" and rc.iters == 0
    assert rc.conv_iter.tolist() == [-1] and np.all(rc.proj == 0)


def test_full_mode_log_has_no_projection_columns():
    H, b, _, z = _problem(L=8, seed=4, K=16)
    s = _solver(H, "f64", tol=1e-10)
    s.set_krylov_log(100000)
    s.solve(b, z, full=True)
    lg = s.krylov_log()
    assert lg.nproj == 0 and lg.rows.shape[0] == lg.n_run
    ci, _ = s.shift_status(z.size)
    rc = s.recalc(z)
    np.testing.assert_array_equal(rc.conv_iter, ci)


def test_recalc_argument_errors():
    s = _solver(w.anderson_3d(4, 2.0, seed=1), "f64")
    with pytest.raises(kw.KomegaError):
        s.recalc([0.1 + 0.1j])                  # no logged solve yet
    with pytest.raises(kw.KomegaError):
        s.recalc([complex("nan")], log=kw.KrylovLog(np.zeros((0, kw.LOG_FIXED), np.complex128),
                                                    np.zeros(0, np.complex128), 1e-10, 0))
    with pytest.raises(kw.KomegaError):
        s.set_krylov_log(-1)
