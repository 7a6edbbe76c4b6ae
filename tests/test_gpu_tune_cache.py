"""GPU: the persistent tuning cache (kw_options.tune_cache).

The product kernel's layout is timed once per context unless a cache file
holds a pick for the same precision, size, sampled-row fingerprint and device:
* the first context times and appends one line; a second context on the same
  operator takes the pick without timing and gives the same bits;
* another operator (same size, other values) misses and appends its own line;
* unreadable lines are skipped, and a stored pick that does not fit the
  operator (lanes that do not exist, or the uniform off-diagonal layout for an
  operator whose off-diagonal values differ) is ignored and timed afresh;
* without a cache every context times.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu

L = 56   # 175,616 rows, 1.23M non-zeros: large enough to be tuned


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()


@pytest.fixture(scope="module")
def ops():
    a = w.anderson_3d(L, 3.0, seed=5)
    b = w.anderson_3d(L, 3.0, seed=6)
    # off-diagonal values that differ: the uniform layout does not apply
    rng = np.random.default_rng(7)
    Hs = a.to_scipy().tocoo()
    off = Hs.row != Hs.col
    upper = off & (Hs.row < Hs.col)
    vals = Hs.data.copy()
    bond = {}
    for r, c, i in zip(Hs.row[upper], Hs.col[upper], np.nonzero(upper)[0]):
        bond[(r, c)] = -1.0 + 0.2 * rng.standard_normal()
        vals[i] = bond[(r, c)]
    for r, c, i in zip(Hs.row[off & ~upper], Hs.col[off & ~upper], np.nonzero(off & ~upper)[0]):
        vals[i] = bond[(c, r)]
    c = w._csr_from_coo(a.m, Hs.row, Hs.col, vals)
    return a, b, c


def _solve(H, prec="df64", cache=None):
    s = kw.Solver(prec, tol=1e-9, maxiter=20, tune_cache=cache)
    s.set_csr(H.rowptr, H.col, H.val)
    bvec = w.gaussian_unit(H.m, 1)
    z = w.shiftk_grid(-8, 8, 16, 0.05)
    r = s.solve(bvec, z, left=np.stack([w.gaussian_unit(H.m, 2)]), check=False)
    return s, r


def _lines(path):
    return [l for l in open(path).read().splitlines() if l.startswith("kwtune1")]


def test_pick_is_stored_and_reused(tmp_path, ops):
    a, b, _ = ops
    path = str(tmp_path / "tune.txt")
    s1, r1 = _solve(a, cache=path)
    st1 = s1.stats()
    assert (st1["tune_runs"], st1["tune_hits"]) == (1, 0)
    assert len(_lines(path)) == 1
    s2, r2 = _solve(a, cache=path)
    st2 = s2.stats()
    assert (st2["tune_runs"], st2["tune_hits"]) == (0, 1)
    assert s2.spmv_config() == s1.spmv_config()
    np.testing.assert_array_equal(r1.proj, r2.proj)
    s3, _ = _solve(b, cache=path)   # other values, other fingerprint
    assert s3.stats()["tune_runs"] == 1
    assert len(_lines(path)) == 2
    s4, _ = _solve(a, prec="f64", cache=path)   # another precision is another key
    assert s4.stats()["tune_runs"] == 1
    assert len(_lines(path)) == 3


def test_bad_lines_and_unfit_picks_are_ignored(tmp_path, ops):
    a, _, c = ops
    path = str(tmp_path / "tune.txt")
    s1, _ = _solve(a, cache=path)
    good = _lines(path)[0].split()
    with open(path, "a") as f:
        f.write("not a tuning line\n")
        f.write("kwtune1 1 2 3\n")
        f.write(" ".join(good[:6] + ["7", good[7]]) + "\n")   # 7 lanes per row does not exist
    s2, _ = _solve(a, cache=path)
    assert s2.stats()["tune_runs"] == 1
    # a stored uniform-layout pick for an operator whose off-diagonal values differ
    s3, r3 = _solve(c, cache=path)
    key = _lines(path)[-1].split()
    with open(path, "a") as f:
        f.write(" ".join(key[:6] + ["65", "0"]) + "\n")
    s4, r4 = _solve(c, cache=path)
    assert s4.stats()["tune_runs"] == 1
    assert s4.spmv_config()[0] < 64
    np.testing.assert_allclose(r4.proj, r3.proj, rtol=0, atol=1e-12 * np.abs(r3.proj).max())


def test_without_a_cache_every_context_times(ops):
    a, _, _ = ops
    for _ in range(2):
        s, _ = _solve(a)
        assert (s.stats()["tune_runs"], s.stats()["tune_hits"]) == (1, 0)
