"""Parity at full size: the benchmark workload (Heisenberg chain N=24, S^z=0,
M=2,704,156, K=1024 shifts w + 0.01i on [-12, 12), b and 3 Gaussian left
vectors, tol 1e-10) in the launch configuration bench.py times.

A full oracle solve at this size is too slow for a test, so the outputs are
checked through quantities the oracle computes one by one:

* x_k for 4 sampled shifts (full mode, same solver settings): the true residual
  ||b - (z_k - H) x_k|| is computed on the CPU with the oracle's CSR product and
  must be within 10 tol (each converged shift's recursive residual is <= tol,
  Eq. 7 and Eq. 19);
* the projections a_l^T x_k of the 1024-shift projected run (Eq. 25-26) must
  agree with a_l^T x_k formed on the CPU from those x_k: both are within
  tol ||a_l|| / dist(z_k, spec) <= tol / Im z_k of the exact value.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLE = np.array([0, 301, 512, 1000])   # band edge, interior, centre (slowest), upper interior


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()
    return w.heisenberg_projected(N=24, K=1024, delta=0.01, tol=1e-10)


@pytest.mark.parametrize("prec", ["df64"])
def test_fullsize_projected_vs_sampled_full_solutions(problem, prec):
    p = problem
    bd = torch.as_tensor(p.b, device="cuda")
    ld = torch.as_tensor(p.left, device="cuda")
    s = kw.Solver(prec, tol=p.tol, maxiter=200000)
    s.set_csr(p.H.rowptr, p.H.col, p.H.val)
    proj = s.solve(bd, p.z, left=ld)                   # the benchmark's solve
    assert proj.status == "KW_OK" and proj.n_converged == p.z.size
    _, res_all = s.shift_status(p.z.size)
    assert np.all(res_all <= p.tol)

    zs = p.z[SAMPLE]
    full = s.solve(bd, zs, left=ld, full=True)
    assert full.status == "KW_OK"
    x = full.x.cpu().numpy()
    Hs = p.H.to_scipy()
    tr = oc.true_residuals(Hs, p.b, zs, x)
    print(f"{prec}: true residuals of the sampled shifts {tr}")
    assert np.all(tr <= 10 * p.tol)

    P = np.vstack([p.b, p.left])
    ref = x @ P.T                                      # a_l^T x_k on the CPU (column 0: b)
    got = proj.proj[SAMPLE]
    bound = 2 * p.tol * np.linalg.norm(P, axis=1)[None, :] / np.abs(zs.imag)[:, None]
    print(f"{prec}: max |projected - a^T x| {np.abs(got - ref).max():.3e} (bound {bound.min():.1e})")
    assert np.all(np.abs(got - ref) <= bound)
    # the full-mode run's own projections are the same numbers
    np.testing.assert_allclose(full.proj, ref, rtol=1e-12, atol=1e-14)


def test_fullsize_recalc_at_midpoints(problem):
    """Sec. 3.3 (iv) at the benchmark size: the 1024-shift DF64 run records its
    Krylov log; the projections at the 1024 midpoints w + dw/2 + 0.01i are
    recomputed from it, and 4 sampled midpoints are re-solved in full mode and
    checked on the CPU (true residual, then a_l^T x against the recalculated
    projections within 2 max(tol, res_k) ||a_l|| / Im z_k)."""
    p = problem
    bd = torch.as_tensor(p.b, device="cuda")
    ld = torch.as_tensor(p.left, device="cuda")
    s = kw.Solver("df64", tol=p.tol, maxiter=200000)
    s.set_csr(p.H.rowptr, p.H.col, p.H.val)
    s.set_krylov_log(200000)
    r = s.solve(bd, p.z, left=ld)
    assert r.status == "KW_OK"
    lg = s.krylov_log()
    assert lg.rows.shape == (r.iters, kw.LOG_FIXED + 1 + p.left.shape[0]) and lg.n_run == r.iters
    zm = p.z + (p.z[1] - p.z[0]).real / 2
    rc = s.recalc(zm)
    print(f"recalc: {rc.n_converged}/{zm.size} midpoints froze within {rc.iters} rows, "
          f"max res {rc.final_res.max():.2e}")
    assert rc.iters == r.iters and rc.n_converged >= 0.95 * zm.size
    zs = zm[SAMPLE]
    full = s.solve(bd, zs, left=ld, full=True)
    assert full.status == "KW_OK"
    x = full.x.cpu().numpy()
    tr = oc.true_residuals(p.H.to_scipy(), p.b, zs, x)
    assert np.all(tr <= 10 * p.tol)
    P = np.vstack([p.b, p.left])
    ref = x @ P.T
    res = np.maximum(rc.final_res[SAMPLE], p.tol)
    bound = 2 * res[:, None] * np.linalg.norm(P, axis=1)[None, :] / np.abs(zs.imag)[:, None]
    print(f"recalc: max |recalc - a^T x| {np.abs(rc.proj[SAMPLE] - ref).max():.3e}")
    assert np.all(np.abs(rc.proj[SAMPLE] - ref) <= bound)


def test_fullsize_anderson_contour_sampled():
    """Anderson L=160 (M=4,096,000, W=4), 2048 real-axis shifts (delta=0.005) and
    2048 contour points, 16 Gaussian left vectors, tol 1e-8, projected mode in the
    FP32-pair form; 4 sampled shifts (including the near-axis circle points, the
    slowest) re-solved in full mode and checked on the CPU."""
    from paper_2001_08707_gb300 import build

    build.build()
    p = w.anderson_contour()
    assert p.H.m == 4096000 and p.z.size == 4096 and p.left.shape == (16, 4096000)
    bd = torch.as_tensor(p.b, device="cuda")
    ld = torch.as_tensor(p.left, device="cuda")
    s = kw.Solver("df64", tol=p.tol, maxiter=300000)
    s.set_csr(p.H.rowptr, p.H.col, p.H.val)
    proj = s.solve(bd, p.z, left=ld)
    print(f"contour: {proj.iters} iterations, status {proj.status}")
    assert proj.status == "KW_OK" and proj.n_converged == p.z.size
    near_axis = 2048 + int(np.argmin(np.abs(p.z[2048:].imag)))
    sample = np.array([5, 1024, 2048 + 512, near_axis])
    zs = p.z[sample]
    full = s.solve(bd, zs, left=ld, full=True)
    assert full.status == "KW_OK"
    x = full.x.cpu().numpy()
    tr = oc.true_residuals(p.H.to_scipy(), p.b, zs, x)
    print(f"contour: true residuals {tr}")
    assert np.all(tr <= 10 * p.tol)
    P = np.vstack([p.b, p.left])
    ref = x @ P.T
    bound = 2 * p.tol * np.linalg.norm(P, axis=1)[None, :] / np.abs(zs.imag)[:, None]
    assert np.all(np.abs(proj.proj[sample] - ref) <= bound)
