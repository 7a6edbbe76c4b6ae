"""Contour-integral eigensolver (contour.py) driven by the oracle's shifted
solves: Table 3 of the Komega paper (L=12 Heisenberg chain, gamma=-5, rho=0.8,
N_z=100, singular values below 1e-3 discarded)."""
import os

import numpy as np
import pytest

from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import contour
from paper_2001_08707_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "heisenberg_L12_table3.txt")


def _table3():
    return np.array([float(l.split()[1]) for l in open(GOLDEN) if l.strip() and not l.startswith("#")])


@pytest.fixture(scope="module")
def chain():
    H = w.heisenberg_chain(12)
    Hs = H.to_scipy()

    def solve(phi, z):
        r = oc.shifted_cocg(Hs, phi, z, tol=1e-12, full=True)
        assert r.status == oc.STATUS_OK
        return r.x

    return H, Hs, solve


@pytest.mark.parametrize("nl", [2, 5])
def test_ss_reproduces_table3(chain, nl):
    H, Hs, solve = chain
    ev, _ = contour.ss_eigs(solve, Hs, H.m, -5.0, 0.8, 100, 10, nl)
    np.testing.assert_allclose(ev, _table3(), atol=6e-7)


def test_ss_single_vector_misses_the_degenerate_partners(chain):
    """SS(10,1): one random vector sees each eigenspace once, so the doubly
    degenerate levels appear once (Table 3 lists five values, NA for n=5, 6)."""
    H, Hs, solve = chain
    ev, _ = contour.ss_eigs(solve, Hs, H.m, -5.0, 0.8, 100, 10, 1)
    np.testing.assert_allclose(ev, np.unique(np.round(_table3(), 6)), atol=6e-7)
