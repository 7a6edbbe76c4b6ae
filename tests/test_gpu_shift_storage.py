"""GPU: FP32 storage of the shifted vectors in full mode (kw_set_shift_storage).

With the option on, x^(k) and p^(k) (Eq. 23-24) are stored and updated as
complex FP32 while the seed recurrence keeps the form's precision, and the
projections come from the projected recurrences (Eq. 25-26) run in the same
solve.  Checks, through the C ABI:

* the seed recurrence is untouched: iteration counts, per-shift convergence
  iterations, final residuals and the projections equal bit for bit those of a
  projected-mode solve of the same form;
* x carries FP32 storage error only.  x_n = x_{n-1} + alpha_n p_n rounds once
  per step and p_n = r_n / pi_n + beta_n p_{n-1} once per step, so after n
  steps the error is of order sqrt(n) eps_32 |x| (eps_32 = 6e-8) for
  rounding that behaves randomly.  Bounds: 2e-6 per shift after 40 steps, and
  for the converged M = 1000 workload (about 2,200 steps) 5e-5 per shift plus
  the convergence term 2 tol / dist(z, spec) of the FP64 comparison;
* the FP32 form ignores the option (its x/p are FP32 already);
* the host-buffer path returns the same complex FP32 x as the device path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense
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


def _solver(H, prec, fp32, **opts):
    s = kw.Solver(prec, **opts)
    s.set_csr(H.rowptr, H.col, H.val)
    s.set_shift_storage(fp32)
    return s


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_seed_recurrence_and_projections_unchanged(prec):
    p = w.anderson_small(L=10, K=64, delta=0.05, tol=1e-10)
    left = w.gaussian_unit(p.H.m, 7, w.STREAM_LEFT, count=2)
    s = _solver(p.H, prec, True, tol=p.tol)
    g = s.solve(p.b, p.z, left=left, full=True)
    ci, fr = s.shift_status(p.z.size)
    assert g.x.dtype == torch.complex64 and tuple(g.x.shape) == (p.z.size, p.H.m)
    ref = _solver(p.H, prec, False, tol=p.tol)
    r = ref.solve(p.b, p.z, left=left, full=False)
    ci_r, fr_r = ref.shift_status(p.z.size)
    assert g.status == r.status == "KW_OK"
    assert g.iters == r.iters and g.n_seed_switch == r.n_seed_switch and g.updates == r.updates
    assert np.array_equal(ci, ci_r) and np.array_equal(fr, fr_r)
    assert np.array_equal(g.proj, r.proj)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_fixed_iterations_x_within_fp32_storage_error(prec):
    p = w.anderson_small(L=12, K=24, delta=0.1)
    n = 40
    orc = oc.shifted_cocg(p.H.to_scipy(), p.b, p.z, tol=0.0, maxiter=n, full=True)
    s = _solver(p.H, prec, True, tol=0.0, maxiter=n)
    g = s.solve(p.b, p.z, full=True)
    assert g.iters == n
    xg = g.x.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(xg - orc.x, axis=1) / np.linalg.norm(orc.x, axis=1)
    print(f"{prec}: max relative x error after {n} steps {err.max():.2e}")
    assert err.max() <= 2e-6
    # the projections are the FP64-class recurrences, as in projected mode
    assert np.abs(g.proj[:, 0] - orc.proj[:, 0]).max() <= 1e-10 * np.abs(orc.proj[:, 0]).max()


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_converged_full_x_against_oracle(prec):
    p = w.anderson_small()
    Hs = p.H.to_scipy()
    orc = oc.shifted_cocg(Hs, p.b, p.z, tol=p.tol, full=True)
    s = _solver(p.H, prec, True, tol=p.tol)
    g = s.solve(p.b, p.z, full=True)
    assert g.status == "KW_OK" and g.n_converged == p.z.size
    xg = g.x.cpu().numpy().astype(np.complex128)
    dist = dense.spectrum_distance(Hs.toarray(), p.z)
    xn = np.linalg.norm(orc.x, axis=1)
    err = np.linalg.norm(xg - orc.x, axis=1)
    print(f"{prec}: max relative x error {np.max(err / xn):.2e}")
    assert np.all(err <= 5e-5 * xn + 2 * p.tol / dist)
    # the spectrum column from the recurrences keeps the FP64-class agreement
    assert np.abs(g.proj[:, 0] - orc.proj[:, 0]).max() <= 1e-10 * np.abs(orc.proj[:, 0]).max()
    # true residual of the FP32 x, computed on the CPU: FP32 storage level
    tr = oc.true_residuals(Hs, p.b, p.z, xg)
    assert np.all(tr <= 1e-4)


def test_fp32_form_ignores_the_option():
    p = w.anderson_small(L=8, K=16, delta=0.1, tol=1e-6)
    a = _solver(p.H, "c32", True, tol=p.tol).solve(p.b, p.z, full=True)
    b = _solver(p.H, "c32", False, tol=p.tol).solve(p.b, p.z, full=True)
    assert a.iters == b.iters
    assert torch.equal(a.x, b.x)
    assert np.array_equal(a.proj, b.proj)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_host_path_and_edges(prec):
    p = w.anderson_small(L=6, K=8, delta=0.2, tol=1e-9)
    s = _solver(p.H, prec, True, tol=p.tol)
    d = s.solve(p.b, p.z, full=True)
    h = s.solve_host(p.H.rowptr, p.H.col, p.H.val, p.b, p.z, full=True)
    assert h.x.dtype == np.complex64
    assert np.array_equal(h.x, d.x.cpu().numpy())
    assert np.array_equal(h.proj, d.proj)
    # one row, one shift: x = b / (z - h)
    H1 = w.CSR(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([0.5]))
    s1 = _solver(H1, prec, True, tol=1e-12)
    g1 = s1.solve(np.array([1.0]), [2.0 + 1.0j], full=True)
    assert abs(complex(g1.x.cpu().numpy()[0, 0]) - 1.0 / (1.5 + 1.0j)) <= 1e-7
    assert abs(g1.proj[0, 0] - 1.0 / (1.5 + 1.0j)) <= 1e-14


@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
@pytest.mark.parametrize("L", [8, 7])
def test_paired_and_single_element_updates_agree(prec, L):
    """With complex FP32 x and p (FP32 storage, or the FP32 form) the x/p
    update takes two adjacent elements per thread (16-byte accesses, each row's
    pairs aligned by the parity of its offset k m) when x starts 16-byte
    aligned, one element otherwise.  The arithmetic per element is the same, so
    an x at an 8-byte offset (single elements) gives the same bits as an
    aligned one (pairs), for even m (512) and odd m (343, where the rows
    alternate parity); the FP64-class seed forms also meet the oracle's bound."""
    tol = 1e-6 if prec == "c32" else 1e-9
    p = w.anderson_small(L=L, K=20, delta=0.1, tol=tol)
    s = _solver(p.H, prec, True, tol=p.tol)
    a = s.solve(p.b, p.z, full=True)
    buf = torch.zeros(p.z.size * p.H.m + 1, dtype=torch.complex64, device="cuda")
    xv = buf[1:].view(p.z.size, p.H.m)
    assert xv.data_ptr() % 16 == 8
    g = s.solve(p.b, p.z, full=True, x_out=xv)
    assert g.iters == a.iters
    assert torch.equal(xv, a.x)
    if prec == "c32":
        return
    Hs = p.H.to_scipy()
    orc = oc.shifted_cocg(Hs, p.b, p.z, tol=p.tol, full=True)
    assert a.status == "KW_OK"
    xg = a.x.cpu().numpy().astype(np.complex128)
    dist = dense.spectrum_distance(Hs.toarray(), p.z)
    err = np.linalg.norm(xg - orc.x, axis=1)
    assert np.all(err <= 5e-5 * np.linalg.norm(orc.x, axis=1) + 2 * p.tol / dist)
