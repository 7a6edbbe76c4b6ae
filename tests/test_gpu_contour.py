"""Contour-integral eigensolver with the CUDA shifted solver: Table 3 of the
Komega paper (L=12 Heisenberg chain, gamma=-5, rho=0.8, N_z=100, SS(10, N_l))."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_08707_gb300 import contour
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "heisenberg_L12_table3.txt")


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_ss_table3_on_gpu(prec):
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    ref = np.array([float(l.split()[1]) for l in open(GOLDEN) if l.strip() and not l.startswith("#")])
    H = w.heisenberg_chain(12)
    solve = contour.gpu_solve_fn(H, prec=prec, tol=1e-12)
    ev, _ = contour.ss_eigs(solve, H.to_scipy(), H.m, -5.0, 0.8, 100, 10, 2)
    np.testing.assert_allclose(ev, ref, atol=6e-7)
    ev1, _ = contour.ss_eigs(solve, H.to_scipy(), H.m, -5.0, 0.8, 100, 10, 1)
    np.testing.assert_allclose(ev1, np.unique(np.round(ref, 6)), atol=6e-7)


@pytest.mark.parametrize("form", ["df64", "df64+x32"])
def test_ss_table3_with_moments_on_gpu(form):
    """The same eigenvalues with the moments formed on the device (kw_shift_combine),
    also from complex-FP32 solutions (FP32 shift storage)."""
    ref = np.array([float(l.split()[1]) for l in open(GOLDEN) if l.strip() and not l.startswith("#")])
    H = w.heisenberg_chain(12)
    mom = contour.gpu_moments_fn(H, prec="df64", tol=1e-12, shift_fp32=form.endswith("x32"))
    ev, _ = contour.ss_eigs(None, H.to_scipy(), H.m, -5.0, 0.8, 100, 10, 2, moments_fn=mom)
    np.testing.assert_allclose(ev, ref, atol=6e-7)


@pytest.mark.parametrize("xdt", ["complex128", "complex64"])
def test_shift_combine_matches_numpy(xdt):
    from paper_2001_08707_gb300 import komega as kw

    rng = np.random.default_rng(3)
    K, m, nk = 131, 1000, 13                     # K not a multiple of the 64-shift weight chunk
    X = (rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))).astype(xdt)
    Wt = rng.standard_normal((nk, K)) + 1j * rng.standard_normal((nk, K))
    s = kw.Solver("f64")
    S = s.shift_combine(torch.as_tensor(X, device="cuda"), Wt).cpu().numpy()
    ref = Wt @ X.astype(np.complex128)
    np.testing.assert_allclose(S, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    one = s.shift_combine(torch.as_tensor(X[:1], device="cuda"), Wt[:1, :1]).cpu().numpy()
    np.testing.assert_allclose(one, Wt[:1, :1] @ X[:1].astype(np.complex128), rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        s.shift_combine(torch.as_tensor(X, device="cuda"), Wt[:, :-1])
    bad = np.zeros((17, K), dtype=np.complex128)        # more than 16 combinations
    with pytest.raises(kw.KomegaError):
        s.shift_combine(torch.as_tensor(X, device="cuda"), bad)
