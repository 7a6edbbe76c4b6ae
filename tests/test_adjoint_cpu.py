"""CPU checks of the input assembly of the differentiable spectrum."""
import numpy as np
import scipy.sparse as sp

from paper_2001_08707_gb300 import adjoint
from paper_2001_08707_gb300 import workloads as w


def test_termset_values_equal_the_summed_matrix():
    j = w.j1j2_chain(10, 1.0, 0.4, 0.2, seed=8)
    ts = adjoint.TermSet(j.terms)
    rng = np.random.default_rng(1)
    for theta in (j.theta, rng.standard_normal(j.theta.size)):
        H = sp.csr_matrix((ts.values(theta), ts.col, ts.rowptr), shape=(ts.m, ts.m)).toarray()
        ref = sum(t * c.to_scipy() for t, c in zip(theta, j.terms)).toarray()
        np.testing.assert_allclose(H, ref, rtol=0, atol=1e-15)
    assert np.all(np.diff(ts.rowptr) >= 1)
