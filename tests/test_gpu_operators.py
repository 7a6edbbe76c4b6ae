"""GPU: operators generated on the fly (kw_set_spin_operator, kw_set_lattice3d).

The references are the generators' CSR matrices of the same Hamiltonians (or,
for shapes the generators do not make, CSR matrices built here element by
element from the definition), applied with scipy in FP64:

* one K1 step q = z_s r - H r, t = r^T q in all three forms with the CSR
  kernel's tolerances: Heisenberg chains (uniform J), the J1-J2 chain with
  random fields (two bond values, fields), a sector away from half filling with
  long-range bonds, cubic and non-cubic Anderson lattices;
* converged solves on the generated operators against the oracle;
* argument errors.
"""
from math import comb

import numpy as np
import pytest
import scipy.sparse as sp

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


def to_pairs(z):
    d = torch.view_as_real(z.to(torch.complex128))
    hi = d.float()
    lo = (d - hi.double()).float()
    return torch.stack([hi[:, 0], lo[:, 0], hi[:, 1], lo[:, 1]], dim=1).contiguous()


def from_pairs(p):
    return torch.complex(p[:, 0].double() + p[:, 1].double(), p[:, 2].double() + p[:, 3].double())


def spin_csr(nsite, nup, bonds, J, h=None):
    """The spin Hamiltonian written out entry by entry (test-side reference)."""
    words = np.array([s for s in range(1 << nsite) if bin(s).count("1") == nup], dtype=np.int64)
    m = words.size
    index = {int(s): i for i, s in enumerate(words)}
    rows, cols, vals = [], [], []
    for i, s in enumerate(words):
        d = 0.0
        for (a, c), Jb in zip(bonds, J):
            if ((s >> a) & 1) == ((s >> c) & 1):
                d += 0.25 * Jb
            else:
                d -= 0.25 * Jb
                rows.append(i)
                cols.append(index[int(s ^ ((1 << a) | (1 << c)))])
                vals.append(0.5 * Jb)
        if h is not None:
            d += sum((0.5 if (s >> k) & 1 else -0.5) * h[k] for k in range(nsite))
        rows.append(i)
        cols.append(i)
        vals.append(d)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


def lattice_csr(nx, ny, nz, eps, hop):
    m = nx * ny * nz
    rows, cols, vals = list(range(m)), list(range(m)), list(eps)
    for i in range(m):
        x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            j = (x + dx) % nx + nx * (((y + dy) % ny) + ny * ((z + dz) % nz))
            rows.append(i)
            cols.append(j)
            vals.append(hop)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


def _chain_bonds(N, d=1):
    return [(i, (i + d) % N) for i in range(N)]


def _j1j2(N, seed):
    mdl = w.j1j2_chain(N, 1.0, 0.4, 0.2, seed=seed)
    th = mdl.theta
    bonds = _chain_bonds(N, 1) + _chain_bonds(N, 2)
    J = [th[0]] * N + [th[1]] * N
    return bonds, J, th[2:], mdl.assemble().to_scipy()


def _set_spin(s, case):
    if case.startswith("heisenberg"):
        N = int(case.split("_N")[1])
        s.set_spin_operator(N, N // 2, _chain_bonds(N), 1.0)
        return w.heisenberg_chain(N).to_scipy()
    if case == "j1j2_N12":
        bonds, J, h, Hs = _j1j2(12, 5)
        s.set_spin_operator(12, 6, bonds, J, h)
        return Hs
    # away from half filling, long-range bonds, one field
    rng = np.random.default_rng(3)
    bonds = [(0, 8), (2, 7), (1, 2), (8, 3), (4, 5), (6, 0), (3, 5)]
    J = rng.uniform(-1, 1, len(bonds))
    h = np.zeros(9)
    h[4] = 0.3
    s.set_spin_operator(9, 4, bonds, J, h)
    return spin_csr(9, 4, bonds, J, h)


def _set_lattice(s, case):
    if case == "anderson_L10":
        H = w.anderson_3d(10, 2.0, seed=1)
        eps = H.to_scipy().diagonal().copy()
        s.set_lattice3d(10, 10, 10, eps, -1.0)
        return H.to_scipy()
    rng = np.random.default_rng(2)
    nx, ny, nz = 4, 5, 3
    eps = rng.uniform(-3, 3, nx * ny * nz)
    s.set_lattice3d(nx, ny, nz, eps, 0.7)
    return lattice_csr(nx, ny, nz, eps, 0.7)


SPIN = ["heisenberg_N8", "heisenberg_N16", "j1j2_N12", "sector_9_4"]
LATTICE = ["anderson_L10", "lattice_4x5x3"]


def _check_step(s, Hs, prec):
    m = Hs.shape[0]
    rng = np.random.default_rng(7)
    r = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    zs = 0.37 - 1.2j
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
    rr = r if prec == "f64" else r.astype(np.complex64).astype(np.complex128)
    q_ref = zs * rr - Hs @ rr
    scale = np.abs(zs) * np.abs(rr) + abs(Hs) @ np.abs(rr)
    tol = 1e-14 if prec == "f64" else 2e-6
    assert np.all(np.abs(q - q_ref) <= tol * scale + 1e-30)
    assert abs(t - np.dot(rr, q_ref)) <= (1e-12 if prec == "f64" else 1e-5) * np.sum(np.abs(rr * q_ref))


@pytest.mark.parametrize("table", [False, True])
@pytest.mark.parametrize("prec", ["f64", "c32", "df64"])
@pytest.mark.parametrize("case", SPIN)
def test_spin_operator_step(case, prec, table):
    s = kw.Solver(prec)
    s.set_spin_table(table)
    Hs = _set_spin(s, case)
    assert s.m == Hs.shape[0]
    _check_step(s, Hs, prec)


@pytest.mark.parametrize("prec", ["f64", "c32", "df64"])
@pytest.mark.parametrize("case", LATTICE)
def test_lattice_operator_step(case, prec):
    s = kw.Solver(prec)
    Hs = _set_lattice(s, case)
    _check_step(s, Hs, prec)


@pytest.mark.parametrize("prec", ["f64", "df64"])
@pytest.mark.parametrize("case", ["heisenberg_N14", "j1j2_N12", "anderson_L10", "j1j2_N12_table"])
def test_generated_operator_converged_solve(case, prec):
    s = kw.Solver(prec, tol=1e-10, maxiter=20000)
    if case.endswith("_table"):
        s.set_spin_table(True)
        case = case[: -len("_table")]
    Hs = _set_lattice(s, case) if case.startswith("anderson") else _set_spin(s, case)
    m = Hs.shape[0]
    b = w.gaussian_unit(m, 31)
    left = np.stack([w.gaussian_unit(m, 32 + i) for i in range(2)])
    lo, hi = (-8.0, 8.0) if case.startswith("anderson") else (-7.0, 3.0)
    z = w.shiftk_grid(lo, hi, 40, 0.05)
    r = s.solve(b, z, left=left)
    ro = oc.shifted_cocg(Hs, b, z, left=left, tol=1e-10, full=False)
    assert r.status == "KW_OK" and abs(r.iters - ro.iters) <= 0.05 * ro.iters + 2
    ev = np.linalg.eigvalsh(Hs.toarray())
    dist = np.array([np.abs(zk - ev).min() for zk in z])
    scale = np.abs(ro.proj).max(axis=0)
    norms = np.linalg.norm(np.vstack([b, left]), axis=1)
    assert np.all(np.abs(r.proj - ro.proj) <= 1e-10 * scale[None, :] + 2e-10 * norms[None, :] / dist[:, None])


def test_spin_table_switch_on_existing_operator():
    """Turning the table on and off for the current operator gives the same product."""
    s = kw.Solver("f64")
    Hs = _set_spin(s, "j1j2_N12")
    rng = np.random.default_rng(3)
    r = torch.as_tensor(rng.standard_normal(Hs.shape[0]) + 1j * rng.standard_normal(Hs.shape[0]), device="cuda")
    qa, qb, qc = torch.empty_like(r), torch.empty_like(r), torch.empty_like(r)
    ta = s.spmv_dot(0.2 + 0.3j, r, qa)
    s.set_spin_table(True)
    tb = s.spmv_dot(0.2 + 0.3j, r, qb)
    s.set_spin_table(False)
    tc = s.spmv_dot(0.2 + 0.3j, r, qc)
    assert (qa - qb).abs().max().item() <= 1e-14 * qa.abs().max().item()
    assert torch.equal(qa, qc) and ta == tc and abs(ta - tb) <= 1e-13 * abs(ta)


def test_generated_operator_argument_errors():
    s = kw.Solver("f64")
    for args in [(32, 16, [(0, 1)], 1.0), (8, 0, [(0, 1)], 1.0), (8, 8, [(0, 1)], 1.0), (8, 4, [(0, 0)], 1.0),
                 (8, 4, [(0, 9)], 1.0), (8, 4, [(0, 1)], float("nan"))]:
        with pytest.raises(kw.KomegaError):
            s.set_spin_operator(*args)
    with pytest.raises(kw.KomegaError):
        s.set_lattice3d(2, 5, 5, np.zeros(50), -1.0)
    with pytest.raises(kw.KomegaError):
        s.set_lattice3d(3, 3, 3, np.zeros(27), float("inf"))
    # the spin sector size C(nsite, nup)
    s.set_spin_operator(10, 3, [(0, 1)], 1.0)
    assert s.m == comb(10, 3)
