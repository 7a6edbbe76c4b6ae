"""GPU: the three-term update with its tiles staged by TMA bulk copies.

With kw_set_bulk_copy(1) K2 (FP32 and FP32-pair forms) stages the tiles of
r_n, q, r_{n-1} and the projection rows in shared memory with cp.async.bulk
copies completed on mbarriers.  A tile is the block and the tiles of a block
are its grid-stride trips, so each thread sums the same elements in the same
order as with plain loads.  The two are separately compiled kernels, and the
FP64 coefficient products of the prologue (and the FP32 form's arithmetic)
may be contracted into FMAs differently in each: they agree to rounding, not
bit for bit.  Checked: agreement after a few iterations at rounding level,
for no full tile (m < 256), exactly whole tiles, a ragged last tile, and
projection counts that select two and three stages; converged solves against
the oracle; the bounded wait, by arming the stages for bytes that never
arrive (the solve ends with KW_ERR_TIMEOUT and the context then solves
correctly).
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


def _chain(m, seed=3):
    """Periodic tight-binding ring with random on-site energies (m rows, 3 per row)."""
    rng = np.random.default_rng(seed)
    i = np.arange(m)
    rows = np.concatenate([i, i, i])
    cols = np.concatenate([i, (i + 1) % m, (i - 1) % m])
    vals = np.concatenate([rng.uniform(-1.0, 1.0, m), -np.ones(m), -np.ones(m)])
    return w._csr_from_coo(m, rows, cols, vals)


def _run(prec, m, nleft, full, bulk, maxiter=3000):
    H = _chain(m)
    b = w.gaussian_unit(m, 21)
    left = np.stack([w.gaussian_unit(m, 22 + i) for i in range(nleft)]) if nleft else None
    z = w.shiftk_grid(-3, 3, 24, 0.04)
    s = kw.Solver(prec, tol=1e-9, maxiter=maxiter)
    s.set_seed_update(0)          # the staged and plain loads of the one-element-per-thread update
    s.set_bulk_copy(bulk)
    s.set_csr(H.rowptr, H.col, H.val)
    r = s.solve(b, z, left=left, full=full, check=False)
    ci, fr = s.shift_status(z.size)
    return r, ci, fr, (None if r.x is None else r.x.cpu().numpy()), (H, b, left, z)


@pytest.mark.parametrize("prec", ["df64", "c32"])
@pytest.mark.parametrize("m,nleft,full", [(200, 2, False), (256, 0, True), (1000, 4, False), (4113, 1, True),
                                          (4113, 8, False), (3072, 16, False), (20001, 4, False)])
def test_staged_update_agrees_with_plain_loads(prec, m, nleft, full):
    a = _run(prec, m, nleft, full, True, maxiter=8)
    b = _run(prec, m, nleft, full, False, maxiter=8)
    ra, rb = a[0], b[0]
    assert (ra.iters, ra.status) == (rb.iters, rb.status) == (8, "KW_NOT_CONVERGED")
    tol = 1e-12 if prec == "df64" else 2e-5
    assert np.abs(ra.proj - rb.proj).max() <= tol * np.abs(rb.proj).max()
    if full:
        assert np.abs(a[3] - b[3]).max() <= tol * np.abs(b[3]).max()
    if m < 256:   # no full tile: both run the plain loop
        np.testing.assert_array_equal(ra.proj, rb.proj)


@pytest.mark.parametrize("m,nleft", [(4113, 4), (3072, 16)])
def test_staged_update_parity_with_oracle(m, nleft):
    r, _, _, _, (H, b, left, z) = _run("df64", m, nleft, False, True)
    assert r.status == "KW_OK"
    ref = oc.shifted_cocg(H.to_scipy(), b, z, left=left, tol=1e-9, full=False)
    # both stop within tol of the exact projections: |a^T (x - x*)| <= tol ||a|| ||b|| / |Im z|
    err = np.abs(r.proj - ref.proj).max(axis=1) * np.abs(z.imag)
    assert err.max() < 4e-9, err.max()


def test_bounded_wait_reports_timeout_and_context_recovers():
    H = _chain(4113)
    b = w.gaussian_unit(H.m, 21)
    z = w.shiftk_grid(-3, 3, 8, 0.04)
    s = kw.Solver("df64", tol=1e-9, maxiter=3000)
    s.set_seed_update(0)
    s.set_bulk_copy(1)
    s.set_csr(H.rowptr, H.col, H.val)
    good = s.solve(b, z)
    s.set_bulk_copy(2)
    bad = s.solve(b, z, check=False)
    assert bad.status == "KW_ERR_TIMEOUT"
    assert bad.iters <= 8
    s.set_bulk_copy(1)
    again = s.solve(b, z)
    assert again.iters == good.iters
    np.testing.assert_array_equal(again.proj, good.proj)


@pytest.mark.parametrize("nleft,staged", [(16, True), (9, True), (8, False), (4, False)])
def test_default_stages_only_many_projection_rows(nleft, staged):
    """With the row-group update off (kw_set_seed_update(0)), the default (-1)
    runs the staged kernel above 9 projection rows (b and nleft left vectors),
    the plain one otherwise: it equals that choice bit for bit."""
    m = 4113
    H = _chain(m)
    b = w.gaussian_unit(m, 21)
    left = np.stack([w.gaussian_unit(m, 22 + i) for i in range(nleft)])
    z = w.shiftk_grid(-3, 3, 24, 0.04)
    out = {}
    for mode in (-1, 1 if staged else 0):
        s = kw.Solver("df64", tol=1e-9, maxiter=8)
        s.set_seed_update(0)
        s.set_bulk_copy(mode)
        s.set_csr(H.rowptr, H.col, H.val)
        out[mode] = s.solve(b, z, left=left, check=False).proj
    np.testing.assert_array_equal(out[-1], out[1 if staged else 0])


def test_bulk_copy_argument():
    s = kw.Solver("df64")
    assert s._lib.kw_set_bulk_copy(s._ctx, 3) == kw.KW_ERR_ARG
    assert s._lib.kw_set_bulk_copy(s._ctx, -2) == kw.KW_ERR_ARG
