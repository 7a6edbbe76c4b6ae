"""CPU pins for the seeded input generators."""
import os
from math import comb

import numpy as np
import pytest

from paper_2001_08707_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "heisenberg_L12_table3.txt")


def _golden_table3():
    vals = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                vals.append(float(line.split()[1]))
    return np.array(vals)


def test_heisenberg_L12_matches_table3():
    """Table 3 of the paper: the seven lowest levels of the L=12 chain (M=924)."""
    H = w.heisenberg_chain(12)
    assert H.m == 924
    d = H.to_scipy().toarray()
    assert np.array_equal(d, d.T)
    e = np.linalg.eigvalsh(d)
    ref = _golden_table3()
    np.testing.assert_allclose(e[: ref.size], ref, atol=6e-7, rtol=0)


@pytest.mark.parametrize("N", [4, 6, 8, 10, 14])
def test_heisenberg_dimension_and_total_spin(N):
    """Sector dimension C(N, N/2); H commutes with S^z (no entry leaves the sector);
    the ground energy of the 4-site ring is -2 J (closed form)."""
    H = w.heisenberg_chain(N)
    assert H.m == comb(N, N // 2)
    d = H.to_scipy().toarray()
    assert np.array_equal(d, d.T)
    # Trace of H: every bond contributes +1/4 (parallel) or -1/4 (antiparallel),
    # averaged over the sector: sum_bonds (P_par - P_anti)/4 with P_anti = N/(2(N-1)).
    p_anti = (N / 2) / (N - 1)
    assert np.isclose(np.trace(d) / H.m, N * ((1 - p_anti) - p_anti) / 4)
    if N == 4:
        assert np.isclose(np.linalg.eigvalsh(d)[0], -2.0)


def test_heisenberg_N20_nnz():
    H = w.heisenberg_chain(20)
    assert H.m == 184756
    j = w.j1j2_chain(20, 1.0, 0.4, 0.2, seed=w.SEED_BASE + 3)
    assert len(j.terms) == 22
    assert j.assemble().nnz == 4074356


def test_j1j2_terms_sum():
    j = w.j1j2_chain(8, 1.0, 0.4, 0.2, seed=3)
    Hsum = sum(t * c.to_scipy() for t, c in zip(j.theta, j.terms)).toarray()
    Ha = j.assemble().to_scipy().toarray()
    np.testing.assert_allclose(Ha, Hsum, atol=1e-15)
    # J2 = 0, h = 0 reduces to the Heisenberg chain
    th = np.zeros_like(j.theta)
    th[0] = 1.0
    np.testing.assert_array_equal(j.assemble(th).to_scipy().toarray(),
                                  w.heisenberg_chain(8).to_scipy().toarray())


def test_anderson_structure():
    L, W = 5, 3.0
    H = w.anderson_3d(L, W, seed=11)
    assert H.m == L ** 3 and H.nnz == 7 * L ** 3
    assert np.all(np.diff(H.rowptr) == 7)
    d = H.to_scipy().toarray()
    assert np.array_equal(d, d.T)
    eps = np.diag(d)
    assert np.all(np.abs(eps) <= W / 2)
    # constant vector: (H 1)_i = eps_i - 6
    np.testing.assert_allclose(d @ np.ones(H.m), eps - 6.0, atol=1e-14)
    for i in range(H.m):
        cols = H.col[H.rowptr[i]:H.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    lo, hi = w.anderson_bounds(W)
    e = np.linalg.eigvalsh(d)
    assert lo <= e[0] and e[-1] <= hi


def test_seeded_reproducible():
    a = w.anderson_small(L=4, K=8)
    b = w.anderson_small(L=4, K=8)
    assert np.array_equal(a.b, b.b) and np.array_equal(a.H.val, b.H.val)
    assert np.isclose(np.linalg.norm(a.b), 1.0)


def test_shift_grids():
    z = w.shiftk_grid(-8.0, 8.0, 64, 0.05)
    assert z[0] == -8.0 + 0.05j
    assert np.isclose(z[-1].real, 8.0 - 16.0 / 64)
    c = w.circle_points(0.3, 0.5, 2048)
    np.testing.assert_allclose(np.abs(c - 0.3), 0.5)
    assert np.isclose(np.min(np.abs(c.imag)), 0.5 * np.sin(np.pi / 2048))


def test_solve_array_checks():
    """The binding checks the sizes the C ABI cannot see before any call."""
    import torch

    from paper_2001_08707_gb300.komega import check_solve_arrays

    m, K = 10, 3
    b = torch.zeros(m, dtype=torch.float64)
    left = torch.zeros(2, m, dtype=torch.float64)
    x = torch.zeros(K, m, dtype=torch.complex128)
    check_solve_arrays(m, b, left, x, K, torch.complex128)
    check_solve_arrays(None, b, None, None, K, torch.complex128)   # no operator yet: nothing to compare
    bad = [dict(b=torch.zeros(m + 1, dtype=torch.float64)),
           dict(left=torch.zeros(2, m - 1, dtype=torch.float64)),
           dict(x=torch.zeros(K, m, dtype=torch.complex64)),
           dict(x=torch.zeros(K + 1, m, dtype=torch.complex128)),
           dict(x=torch.zeros(m, K, dtype=torch.complex128).t())]
    for case in bad:
        args = dict(b=b, left=left, x=x)
        args.update(case)
        with pytest.raises(ValueError):
            check_solve_arrays(m, args["b"], args["left"], args["x"], K, torch.complex128)


def test_vector_byte_checks():
    import torch

    from paper_2001_08707_gb300.komega import check_vector_bytes

    m = 7
    check_vector_bytes("r", torch.zeros(m, dtype=torch.complex128), m, 16)
    check_vector_bytes("r", torch.zeros(m, 4, dtype=torch.float32), m, 16)   # FP32 pairs
    check_vector_bytes("r", torch.zeros(m, dtype=torch.complex64), m, 8)
    for bad in (torch.zeros(m + 1, dtype=torch.complex128), torch.zeros(m, dtype=torch.complex64),
                torch.zeros(4, m, dtype=torch.float32).t()):
        with pytest.raises(ValueError):
            check_vector_bytes("r", bad, m, 16)
