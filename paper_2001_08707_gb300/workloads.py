"""Seeded synthetic inputs for the shifted Krylov problem (z_k I - H) x^(k) = b.

This module builds inputs only: sparse Hamiltonians in CSR form, right-hand
sides, left (projection) vectors and shift grids.  It contains none of the
solver's arithmetic, so both the CUDA path and the CPU oracle consume exactly
the same arrays without sharing any solver code.

Models
------
* 3D Anderson tight-binding model on an L x L x L periodic cube: hopping -1
  to the six nearest neighbours, on-site energies uniform on [-W/2, W/2].
  Site index i = x + L*(y + L*z); columns sorted in every row; the diagonal is
  always stored (7 non-zeros per row for L >= 3).
* Spin-1/2 Heisenberg chain H = J sum_i S_i . S_{i+1} with periodic boundary
  (the model of Eq. 41 of the Komega paper, Sec. 4.1), restricted to the
  S^z_total = 0 sector.  Basis: N-bit words with N/2 set bits (bit i = spin up
  on site i) in increasing integer order.  Diagonal: +J/4 for a parallel bond,
  -J/4 for an antiparallel one; off-diagonal: +J/2 between two words that
  differ by exchanging an antiparallel neighbour pair.
* J1-J2 chain with site fields: H = J1 H_1 + J2 H_2 + sum_i h_i S^z_i, where
  H_1 holds the nearest-neighbour bonds, H_2 the next-nearest bonds (i, i+2),
  and S^z_i is diagonal with entries +-1/2.  The term matrices are returned
  separately for the parameter derivative.

Shift grids follow the ShiftK convention of the paper (Sec. 3.2.2):
omega_i = omega_min + i (omega_max - omega_min) / n, i = 0..n-1, and circle
points for contour integrals z_j = gamma + rho exp[2 pi i (j + 1/2) / N_z]
(Sec. 4.1).

Random numbers come from numpy's PCG64 (``numpy.random.default_rng``) seeded
with ``[seed, stream]`` so that every array has its own reproducible stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Stream identifiers for default_rng([seed, stream]).
STREAM_DISORDER = 1
STREAM_RHS = 2
STREAM_LEFT = 3
STREAM_FIELDS = 4
STREAM_BATCH = 5
STREAM_PERTURB = 6


@dataclass
class CSR:
    """Real square sparse matrix in CSR form (int64 rowptr, int32 col, f64 val)."""

    m: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.m, self.m))


def _csr_from_coo(m: int, rows, cols, vals) -> CSR:
    """Assemble CSR with duplicates summed and columns sorted within each row."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * np.int64(m) + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size:
        key_new = np.ones(rows.size, dtype=bool)
        key_new[1:] = key[1:] != key[:-1]
        if key_new.all():
            counts = np.bincount(rows, minlength=m)
            rowptr = np.zeros(m + 1, dtype=np.int64)
            np.cumsum(counts, out=rowptr[1:])
            return CSR(m, rowptr, cols.astype(np.int32), vals)
        seg = np.cumsum(key_new) - 1
        nuniq = int(seg[-1]) + 1
        v = np.zeros(nuniq, dtype=np.float64)
        np.add.at(v, seg, vals)
        rows, cols, vals = rows[key_new], cols[key_new], v
    counts = np.bincount(rows, minlength=m)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(m, rowptr, cols.astype(np.int32), vals)


# --------------------------------------------------------------------------
# 3D Anderson model
# --------------------------------------------------------------------------
def anderson_3d(L: int, W: float, seed: int, hopping: float = -1.0) -> CSR:
    """Periodic L^3 Anderson model; on-site energies uniform on [-W/2, W/2]."""
    if L < 3:
        raise ValueError("Anderson cube needs L >= 3 so that the six neighbours are distinct")
    rng = np.random.default_rng([seed, STREAM_DISORDER])
    m = L * L * L
    eps = rng.uniform(-W / 2.0, W / 2.0, size=m)
    i = np.arange(m, dtype=np.int64)
    x = i % L
    y = (i // L) % L
    z = i // (L * L)
    neigh = []
    for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        neigh.append(((x + dx) % L) + L * (((y + dy) % L) + L * ((z + dz) % L)))
    rows = np.concatenate([i] + [i] * 6)
    cols = np.concatenate([i] + neigh)
    vals = np.concatenate([eps] + [np.full(m, hopping)] * 6)
    return _csr_from_coo(m, rows, cols, vals)


def anderson_bounds(W: float, hopping: float = -1.0) -> tuple[float, float]:
    """Gershgorin interval of the 3D Anderson model: +-(6|t| + W/2)."""
    r = 6.0 * abs(hopping) + W / 2.0
    return -r, r


# --------------------------------------------------------------------------
# Spin chains in the S^z = 0 sector
# --------------------------------------------------------------------------
def _popcount(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.uint64)
    c = np.zeros(a.shape, dtype=np.int64)
    while True:
        nz = a != 0
        if not nz.any():
            return c
        c += nz
        a = a & (a - np.uint64(1)) * nz.astype(np.uint64)


def sz0_basis(N: int) -> np.ndarray:
    """All N-bit words with N/2 set bits, increasing (the S^z_total = 0 basis)."""
    if N % 2 or N < 2 or N > 40:
        raise ValueError("N must be even, 2 <= N <= 40")
    words = np.arange(1 << N, dtype=np.int64)
    return words[_popcount(words) == N // 2]


def _bond_terms(N: int, basis: np.ndarray, bonds):
    """COO entries of sum over bonds of S_i . S_j (J = 1) on the given basis."""
    m = basis.size
    idx = np.arange(m, dtype=np.int64)
    diag = np.zeros(m, dtype=np.float64)
    rows, cols = [], []
    for (i, j) in bonds:
        bi = (basis >> i) & 1
        bj = (basis >> j) & 1
        anti = bi != bj
        diag += np.where(anti, -0.25, 0.25)
        flipped = basis[anti] ^ ((1 << i) | (1 << j))
        rows.append(idx[anti])
        cols.append(np.searchsorted(basis, flipped))
    r = np.concatenate([idx] + rows)
    c = np.concatenate([idx] + cols)
    v = np.concatenate([diag] + [np.full(x.size, 0.5) for x in rows])
    return r, c, v


def heisenberg_chain(N: int, J: float = 1.0) -> CSR:
    """Periodic spin-1/2 Heisenberg chain H = J sum_i S_i . S_{i+1}, S^z = 0."""
    if N < 4:
        raise ValueError("chain needs N >= 4")
    basis = sz0_basis(N)
    r, c, v = _bond_terms(N, basis, [(i, (i + 1) % N) for i in range(N)])
    return _csr_from_coo(basis.size, r, c, J * v)


@dataclass
class J1J2Model:
    """H(theta) = sum_m theta_m H_m with theta = (J1, J2, h_0, ..., h_{N-1})."""

    N: int
    theta: np.ndarray
    terms: list = field(default_factory=list)  # list of CSR, one per parameter

    def assemble(self, theta: np.ndarray | None = None) -> CSR:
        th = self.theta if theta is None else np.asarray(theta, dtype=np.float64)
        m = self.terms[0].m
        rows, cols, vals = [], [], []
        for t, c in zip(th, self.terms):
            rr = np.repeat(np.arange(m, dtype=np.int64), np.diff(c.rowptr))
            rows.append(rr)
            cols.append(c.col.astype(np.int64))
            vals.append(t * c.val)
        return _csr_from_coo(m, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def j1j2_chain(N: int, J1: float, J2: float, hmax: float, seed: int) -> J1J2Model:
    """Periodic J1-J2 chain with random fields h_i uniform on [-hmax, hmax]."""
    if N < 5:
        raise ValueError("J1-J2 chain needs N >= 5")
    rng = np.random.default_rng([seed, STREAM_FIELDS])
    h = rng.uniform(-hmax, hmax, size=N)
    basis = sz0_basis(N)
    m = basis.size
    terms = []
    for bonds in ([(i, (i + 1) % N) for i in range(N)], [(i, (i + 2) % N) for i in range(N)]):
        terms.append(_csr_from_coo(m, *_bond_terms(N, basis, bonds)))
    idx = np.arange(m, dtype=np.int64)
    for i in range(N):
        sz = np.where((basis >> i) & 1, 0.5, -0.5)
        terms.append(_csr_from_coo(m, idx, idx, sz))
    theta = np.concatenate([[J1, J2], h])
    return J1J2Model(N, theta, terms)


def chain_bounds(csr: CSR) -> tuple[float, float]:
    """Gershgorin interval of a CSR matrix."""
    rows = np.repeat(np.arange(csr.m), np.diff(csr.rowptr))
    diag = np.zeros(csr.m)
    off = np.zeros(csr.m)
    on = csr.col == rows
    np.add.at(diag, rows[on], csr.val[on])
    np.add.at(off, rows[~on], np.abs(csr.val[~on]))
    return float((diag - off).min()), float((diag + off).max())


# --------------------------------------------------------------------------
# Vectors and shifts
# --------------------------------------------------------------------------
def gaussian_unit(m: int, seed: int, stream: int = STREAM_RHS, count: int | None = None) -> np.ndarray:
    """Seeded Gaussian vector(s) normalised to unit 2-norm (shape [m] or [count, m])."""
    rng = np.random.default_rng([seed, stream])
    n = 1 if count is None else count
    v = rng.standard_normal((n, m))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v[0] if count is None else v


def shiftk_grid(omega_min: float, omega_max: float, n: int, delta: float) -> np.ndarray:
    """ShiftK frequency grid omega_i = omega_min + i (omega_max - omega_min)/n, plus i*delta."""
    i = np.arange(n, dtype=np.float64)
    return (omega_min + i * (omega_max - omega_min) / n) + 1j * delta


def circle_points(gamma: float, rho: float, nz: int) -> np.ndarray:
    """Contour points z_j = gamma + rho exp[2 pi i (j + 1/2) / N_z]."""
    j = np.arange(nz, dtype=np.float64)
    return gamma + rho * np.exp(2j * np.pi * (j + 0.5) / nz)


# --------------------------------------------------------------------------
# The named workloads
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    H: CSR
    b: np.ndarray            # real [m], unit norm
    z: np.ndarray            # complex [K]
    left: np.ndarray | None  # real [L, m] or None
    tol: float
    full: bool               # True: return x^(k); False: projections only
    extra: dict = field(default_factory=dict)


SEED_BASE = 2001087


def anderson_small(L: int = 10, K: int = 64, delta: float = 0.05, seed: int = SEED_BASE + 0,
                   tol: float = 1e-10) -> Problem:
    """Anderson cube (default L=10, M=1000) with on-site U[-1,1], K shifts on [-8, 8]."""
    H = anderson_3d(L, 2.0, seed)
    b = gaussian_unit(H.m, seed)
    z = shiftk_grid(-8.0, 8.0, K, delta)
    return Problem(f"anderson_L{L}_K{K}_full", H, b, z, None, tol, True)


def heisenberg_projected(N: int = 24, K: int = 1024, delta: float = 0.01, n_gauss: int = 3,
                         seed: int = SEED_BASE + 1, tol: float = 1e-10) -> Problem:
    """Heisenberg chain (N=24: M=2,704,156), K shifts on [-12, 12]; left = {b, 3 Gaussians}."""
    H = heisenberg_chain(N)
    b = gaussian_unit(H.m, seed)
    g = gaussian_unit(H.m, seed, STREAM_LEFT, count=n_gauss)
    left = np.vstack([b[None, :], g])
    z = shiftk_grid(-12.0, 12.0, K, delta)
    return Problem(f"heisenberg_N{N}_K{K}_proj{left.shape[0]}", H, b, z, left, tol, False)


def anderson_batch(n: int = 48, L_range=(16, 48), W_range=(2.0, 16.0), K_range=(32, 512),
                   delta_range=(0.02, 0.1), seed: int = SEED_BASE + 2, tol: float = 1e-8) -> list:
    """n independent Anderson cubes of uneven size: L integer-uniform in L_range,
    disorder W uniform in W_range, K integer-uniform in K_range shifts on the
    cube's Gershgorin interval +-0.5 with delta uniform in delta_range; each with
    its own seeded b; full x returned."""
    rng = np.random.default_rng([seed, STREAM_BATCH])
    out = []
    for i in range(n):
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        W = float(rng.uniform(*W_range))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        delta = float(rng.uniform(*delta_range))
        H = anderson_3d(L, W, seed * 1000 + i)
        b = gaussian_unit(H.m, seed * 1000 + i)
        lo, hi = anderson_bounds(W)
        z = shiftk_grid(lo - 0.5, hi + 0.5, K, delta)
        out.append(Problem(f"anderson_batch{i}_L{L}_K{K}", H, b, z, None, tol, True,
                           {"L": L, "W": W, "delta": delta}))
    return out


def anderson_contour(L: int = 160, W: float = 4.0, n_real: int = 2048, n_circle: int = 2048,
                     n_left: int = 16, seed: int = SEED_BASE + 4, tol: float = 1e-8) -> Problem:
    """Anderson cube (L=160: M=4,096,000), 16 Gaussian left vectors, real-axis + circle shifts."""
    H = anderson_3d(L, W, seed)
    b = gaussian_unit(H.m, seed)
    left = gaussian_unit(H.m, seed, STREAM_LEFT, count=n_left)
    lo, hi = anderson_bounds(W)
    z = np.concatenate([shiftk_grid(lo - 0.5, hi + 0.5, n_real, 0.005),
                        circle_points(0.3, 0.5, n_circle)])
    return Problem(f"anderson_L{L}_K{z.size}_proj{n_left}", H, b, z, left, tol, False)
