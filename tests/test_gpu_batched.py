"""Batched solves (kw_solve_batched): many uneven problems in one captured graph.

* A batch gives, instance by instance, exactly the results of kw_solve on the
  same inputs (same kernels, deterministic reductions).
* Every instance agrees with the oracle within the convergence bound.
* Full size: 48 Anderson cubes, L in {16..48} (M 4,096-110,592), W in [2, 16],
  K in {32..512}, delta in [0.02, 0.1], tol 1e-8, full x; two sampled shifts
  per instance checked through true residuals on the CPU.
"""
import numpy as np
import pytest

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


def _small_batch():
    probs = w.anderson_batch(n=6, L_range=(4, 7), K_range=(5, 40), seed=77)
    out = []
    for i, p in enumerate(probs):
        d = {"H": p.H, "b": p.b, "z": p.z, "tol": p.tol, "full": i % 3 != 2}
        if i % 2:
            d["left"] = w.gaussian_unit(p.H.m, i, w.STREAM_LEFT, count=2)
        out.append(d)
    return out


@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
def test_batched_equals_individual_solves(prec):
    """Each instance of the batch ends exactly as its own solve.  (The FP32-vector
    form stalls on some of these instances and may end in a reported breakdown
    after thousands of iterations; the batch must then report the same.)"""
    batch = _small_batch()
    s = kw.Solver(prec, maxiter=20000)
    res = s.solve_batched(batch, check=prec != "c32")
    for d, r in zip(batch, res):
        one = kw.Solver(prec, maxiter=20000, tol=d["tol"])
        one.set_csr(d["H"].rowptr, d["H"].col, d["H"].val)
        g = one.solve(d["b"], d["z"], left=d.get("left"), full=d["full"], check=prec != "c32")
        assert r.iters == g.iters and r.status == g.status and r.n_seed_switch == g.n_seed_switch
        np.testing.assert_array_equal(r.proj, g.proj)
        if d["full"]:
            np.testing.assert_array_equal(r.x.cpu().numpy(), g.x.cpu().numpy())


def test_batched_matches_oracle():
    batch = _small_batch()
    res = kw.Solver("f64", maxiter=20000).solve_batched(batch)
    for d, r in zip(batch, res):
        orc = oc.shifted_cocg(d["H"].to_scipy(), d["b"], d["z"], left=d.get("left"), tol=d["tol"], full=d["full"])
        assert r.status == "KW_OK"
        allow = 2 * d["tol"] / np.abs(d["z"].imag)[:, None]
        assert np.all(np.abs(r.proj - orc.proj) <= 1e-10 * np.abs(orc.proj).max(axis=0)[None, :] + allow)


def test_batched_reports_per_instance_status():
    """With an iteration cap some instances stop unconverged; each instance's
    status and iteration count are those of its own solve under the same cap."""
    batch = _small_batch()
    res = kw.Solver("f64", maxiter=60).solve_batched(batch, check=False)
    statuses = set()
    for d, r in zip(batch, res):
        one = kw.Solver("f64", maxiter=60, tol=d["tol"])
        one.set_csr(d["H"].rowptr, d["H"].col, d["H"].val)
        g = one.solve(d["b"], d["z"], left=d.get("left"), full=d["full"], check=False)
        assert (r.status, r.iters, r.n_converged) == (g.status, g.iters, g.n_converged)
        statuses.add(r.status)
    assert "KW_NOT_CONVERGED" in statuses


@pytest.mark.slow
def test_fullsize_batch_of_48():
    probs = w.anderson_batch()
    assert len(probs) == 48
    ms = [p.H.m for p in probs]
    assert min(ms) >= 16 ** 3 and max(ms) <= 48 ** 3
    batch = [{"H": p.H, "b": p.b, "z": p.z, "tol": p.tol, "full": True} for p in probs]
    res = kw.Solver("df64", maxiter=200000).solve_batched(batch)
    iters = [r.iters for r in res]
    print(f"batch of 48: iterations min {min(iters)} max {max(iters)}, "
          f"shift-row updates {sum(r.updates * p.H.m for r, p in zip(res, probs)):.3e}")
    for p, r in zip(probs, res):
        assert r.status == "KW_OK" and r.n_converged == p.z.size
        ks = np.array([0, p.z.size // 2])
        x = r.x[ks].cpu().numpy()
        tr = oc.true_residuals(p.H.to_scipy(), p.b, p.z[ks], x)
        assert np.all(tr <= 10 * p.tol), (p.name, tr)
