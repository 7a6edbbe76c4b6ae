"""GPU: the two iteration schedules give the same numbers.

With stream overlap (the default) the shift scalars of iteration n run beside
the product of iteration n+1, and a seed switch reaches that product through
the next three-term update by linearity; on one stream the kernels run in
order.  The arithmetic is the same, so every output must agree bit for bit,
in all three forms, projected and full, with many seed switches, and for the
callback operator.
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


def _run(prec, overlap, full, op="csr"):
    H = w.anderson_3d(9, 3.0, seed=4)
    b = w.gaussian_unit(H.m, 5)
    left = np.stack([w.gaussian_unit(H.m, 6 + i) for i in range(3)])
    z = w.shiftk_grid(-8, 8, 40, 0.03)
    s = kw.Solver(prec, tol=1e-9, maxiter=3000)
    s.set_stream_overlap(overlap)
    if op == "csr":
        s.set_csr(H.rowptr, H.col, H.val)
    else:
        s.set_lattice3d(9, 9, 9, H.to_scipy().diagonal().copy(), -1.0)
    r = s.solve(b, z, left=left, full=full, check=False)
    ci, fr = s.shift_status(z.size)
    x = None if r.x is None else r.x.cpu().numpy()
    return r, ci, fr, x


@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
def test_overlap_and_single_stream_agree_bitwise(prec, full):
    a = _run(prec, True, full)
    b = _run(prec, False, full)
    ra, rb = a[0], b[0]
    assert (ra.iters, ra.status, ra.n_seed_switch, ra.updates) == (rb.iters, rb.status, rb.n_seed_switch, rb.updates)
    assert ra.n_seed_switch > 10
    np.testing.assert_array_equal(ra.proj, rb.proj)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    if full:
        np.testing.assert_array_equal(a[3], b[3])


def test_overlap_agrees_for_generated_operator():
    a = _run("df64", True, False, op="lattice")
    b = _run("df64", False, False, op="lattice")
    np.testing.assert_array_equal(a[0].proj, b[0].proj)
    assert a[0].iters == b[0].iters


def test_stream_overlap_argument():
    s = kw.Solver("f64")
    assert s._lib.kw_set_stream_overlap(s._ctx, 2) == kw.KW_ERR_ARG
