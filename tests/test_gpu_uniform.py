"""GPU: the uniform off-diagonal SpMV layout (kw_set_spmv_config(64 + G)).

Every off-diagonal entry of the lattice operators has one value (Anderson
hopping -1, Heisenberg spin-flip J/2); the layout keeps only int32 offsets, the
off-diagonal columns and the summed diagonal.  Checks, through the C ABI:

* q = z_s r - H r and t = r^T q for G = 1..16, and for the layout's SELL-32
  copy (config 96: slot-major columns of 32-row slices), in all three forms on
  lattice operators and on ragged uniform matrices (empty rows, rows without a
  diagonal, a diagonal split into two entries, a diagonal-only matrix, 1x1),
  with the tolerances of the CSR kernel's parity test;
* forcing the layout on an operator with two off-diagonal values fails with
  KW_ERR_ARG, and so does forcing the SELL-32 copy where its padding would
  exceed three times the columns;
* converged solves on the layout agree with the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu
UNIFORM = 64


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()


def to_pairs(z):
    d = torch.view_as_real(z.to(torch.complex128))
    hi = d.float()
    lo = (d - hi.double()).float()
    return torch.stack([hi[:, 0], lo[:, 0], hi[:, 1], lo[:, 1]], dim=1).contiguous()


def from_pairs(p):
    return torch.complex(p[:, 0].double() + p[:, 1].double(), p[:, 2].double() + p[:, 3].double())


def _uniform_ragged(m, density, seed, v, no_diag=(), split_diag=(), empty=()):
    """Symmetric pattern, every off-diagonal value v, random diagonal; some rows
    without a diagonal entry, some with it split into two entries, some empty."""
    import scipy.sparse as sp

    rng = np.random.default_rng(seed)
    A = sp.random(m, m, density=density, random_state=rng, format="coo")
    pat = set()
    for i, j in zip(A.row, A.col):
        if i != j and i not in empty and j not in empty:
            pat.add((i, j))
            pat.add((j, i))
    rows = [[] for _ in range(m)]
    for i, j in pat:
        rows[i].append((j, v))
    d = rng.uniform(-2, 2, m)
    for i in range(m):
        if i in empty or i in no_diag:
            continue
        if i in split_diag:
            rows[i] += [(i, 0.25 * d[i]), (i, 0.75 * d[i])]
        else:
            rows[i].append((i, d[i]))
    rowptr = np.zeros(m + 1, np.int64)
    col, val = [], []
    for i in range(m):
        ent = sorted(rows[i], key=lambda e: e[0])
        col += [e[0] for e in ent]
        val += [e[1] for e in ent]
        rowptr[i + 1] = len(col)
    return w.CSR(m, rowptr, np.array(col, np.int32), np.array(val, np.float64))


CASES = {
    "anderson_L10": lambda: w.anderson_3d(10, 2.0, seed=1),
    "heisenberg_N12": lambda: w.heisenberg_chain(12),
    "ragged_4097": lambda: _uniform_ragged(4097, 0.002, 3, 0.7, no_diag=(5, 6, 4096), split_diag=(7, 100),
                                           empty=(0, 17)),
    "ragged_33": lambda: _uniform_ragged(33, 0.2, 4, -1.0, no_diag=(0,), split_diag=(32,)),
    "diagonal_only": lambda: w.CSR(5, np.arange(6, dtype=np.int64), np.arange(5, dtype=np.int32),
                                   np.array([1.0, -2.0, 0.3, 0.0, 4.5])),
    "one_by_one": lambda: w.CSR(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([2.5])),
}


@pytest.mark.parametrize("G", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("prec", ["f64", "c32", "df64"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_uniform_spmv_dot(case, prec, G):
    H = CASES[case]()
    Hs = H.to_scipy()
    rng = np.random.default_rng(7)
    r = rng.standard_normal(H.m) + 1j * rng.standard_normal(H.m)
    zs = 0.37 - 1.2j
    s = kw.Solver(prec)
    s.set_spmv_config(UNIFORM + G, -1)
    s.set_csr(H.rowptr, H.col, H.val)
    assert s.spmv_config()[0] == UNIFORM + G
    if prec == "df64":
        rd = to_pairs(torch.as_tensor(r, device="cuda"))
        qd = torch.empty_like(rd)
        t = s.spmv_dot(zs, rd, qd)
        q = from_pairs(qd).cpu().numpy()
        r64 = from_pairs(rd).cpu().numpy()
        q_ref = zs * r64 - Hs @ r64
        scale = np.abs(zs) * np.abs(r64) + abs(Hs) @ np.abs(r64)
        assert np.all(np.abs(q - q_ref) <= 1e-13 * scale)
        assert abs(t - np.dot(r64, q_ref)) <= 1e-12 * np.sum(np.abs(r64 * q_ref))
        return
    dt = torch.complex128 if prec == "f64" else torch.complex64
    rd = torch.as_tensor(r, device="cuda").to(dt)
    qd = torch.empty_like(rd)
    t = s.spmv_dot(zs, rd, qd)
    q = qd.cpu().numpy().astype(np.complex128)
    if prec == "f64":
        q_ref = zs * r - Hs @ r
        scale = np.abs(zs) * np.abs(r) + abs(Hs) @ np.abs(r)
        assert np.all(np.abs(q - q_ref) <= 1e-15 * 8 * scale)
        assert abs(t - np.dot(r, q_ref)) <= 1e-12 * np.sum(np.abs(r * q_ref))
    else:
        r32 = r.astype(np.complex64).astype(np.complex128)
        q_ref = zs * r32 - Hs @ r32
        scale = np.abs(zs) * np.abs(r32) + abs(Hs) @ np.abs(r32)
        assert np.all(np.abs(q - q_ref) <= 2e-6 * scale + 1e-30)
        assert abs(t - np.dot(r32, q_ref)) <= 1e-5 * np.sum(np.abs(r32 * q_ref))


def test_forcing_uniform_on_two_valued_operator_fails():
    H = w.j1j2_chain(10, 1.0, 0.4, 0.0, seed=5).assemble()    # off-diagonals J1/2 and J2/2
    s = kw.Solver("f64")
    s.set_spmv_config(UNIFORM + 1, -1)
    s.set_csr(H.rowptr, H.col, H.val)
    with pytest.raises(kw.KomegaError) as ei:
        s.solve(w.gaussian_unit(H.m, 1), [0.1 + 0.1j])
    assert ei.value.status == kw.KW_ERR_ARG


def test_forcing_uniform_sell_with_heavy_padding_fails():
    # a star: row 0 couples to the 63 others, so slice 0 needs 63 slots for 32 rows
    m = 64
    rows = [[(j, -1.0) for j in range(1, m)]] + [[(0, -1.0)] for _ in range(1, m)]
    rowptr = np.zeros(m + 1, np.int64)
    col, val = [], []
    for i in range(m):
        col += [c for c, _ in rows[i]]
        val += [v for _, v in rows[i]]
        rowptr[i + 1] = len(col)
    H = w.CSR(m, rowptr, np.array(col, np.int32), np.array(val, np.float64))
    s = kw.Solver("f64")
    s.set_spmv_config(UNIFORM + 32, -1)
    s.set_csr(H.rowptr, H.col, H.val)
    with pytest.raises(kw.KomegaError) as ei:
        s.solve(w.gaussian_unit(H.m, 1), [0.1 + 0.1j])
    assert ei.value.status == kw.KW_ERR_ARG
    s.set_spmv_config(UNIFORM + 1, -1)          # the row-per-thread form of the layout still works
    r = s.solve(w.gaussian_unit(H.m, 1), [0.1 + 0.1j])
    assert r.status == "KW_OK"


@pytest.mark.parametrize("layout", [UNIFORM + 1, UNIFORM + 32])
@pytest.mark.parametrize("prec", ["f64", "df64"])
@pytest.mark.parametrize("case", ["anderson_L10", "heisenberg_N12"])
def test_uniform_converged_solve_matches_oracle(case, prec, layout):
    H = CASES[case]()
    Hs = H.to_scipy()
    b = w.gaussian_unit(H.m, 21)
    left = np.stack([w.gaussian_unit(H.m, 22 + i) for i in range(2)])
    lo, hi = w.chain_bounds(H) if case.startswith("heis") else (-8.0, 8.0)
    z = w.shiftk_grid(lo, hi, 48, 0.05)
    s = kw.Solver(prec, tol=1e-10, maxiter=20000)
    s.set_spmv_config(layout, -1)
    s.set_csr(H.rowptr, H.col, H.val)
    r = s.solve(b, z, left=left)
    ro = oc.shifted_cocg(Hs, b, z, left=left, tol=1e-10, full=False)
    assert r.status == "KW_OK" and abs(r.iters - ro.iters) <= 0.05 * ro.iters + 2
    ev = np.linalg.eigvalsh(Hs.toarray())
    dist = np.array([np.abs(zk - ev).min() for zk in z])
    scale = np.abs(ro.proj).max(axis=0)
    norms = np.linalg.norm(np.vstack([b, left]), axis=1)
    bound = 1e-10 * scale[None, :] + 2e-10 * norms[None, :] / dist[:, None]
    assert np.all(np.abs(r.proj - ro.proj) <= bound)
