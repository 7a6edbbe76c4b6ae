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
